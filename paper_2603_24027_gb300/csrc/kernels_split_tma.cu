// kernels_split_tma.cu -- half-step kernels with TMA-staged planes.
//
// The four half-steps of the method, each an in-place update of one family
// of arrays that reads only arrays it does not write (as in kernels_step.cu):
//   k_sfwd_h  Ht^{n+1/2} = Ht^{n-1/2} - S curlE(E^n)            (+ psi_H)
//   k_sfwd_e  E^{n+1} = E^n + cb (curlH(Ht^{n+1/2}) - J)         (+ psi_E, objective)
//   k_srev_e  E^n = E^{n+1} - cb (curlH Ht^{n+1/2} - J) on the interior, dL/dcb,
//             lam_H += transpose of the E half-step               (+ lam_psi_E)
//   k_srev_h  Ht^{n-1/2} = Ht^{n+1/2} + S curlE E^n on the interior,
//             lam_E += transpose of the H half-step               (+ lam_psi_H)
// A CTA owns a 32 x TY column tile and a z chunk [k0, k1).  The planes it
// reads (k0-1 .. k1 at most) stream through an S-stage ring: "halo" boxes cover x in [x0-4, x0+36),
// y in [y0-1, y0+TY+1) (neighbours at +-1), "own" boxes the tile itself.
// Out-of-grid box elements arrive as zeros (the zero-padding boundary).  The
// CPML auxiliaries are staged only for tiles/planes inside an absorbing slab.
// Per-cell arithmetic matches kernels_step.cu operation for operation.
#include <cudaTypedefs.h>

#include "fdtd_internal.cuh"
#include "tma.cuh"

namespace fdtd {

template <int TY>
struct SL {
  static constexpr int HW = 40, HR = TY + 2, HP = HW * HR;   // halo box plane (floats)
  static constexpr int OW = 32, OR = TY, OP = OW * OR;       // own box plane
  static constexpr int r128(int b) { return (b + 127) / 128 * 128; }
};

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

// ------------------------------------------------------------ pipeline ---
// Ring over planes p0..p1.  Plane p lives in stage (p - p0) % S; its barrier
// completes once per use, parity ((p - p0) / S) & 1.  Every issued plane must
// be waited for before its stage is re-armed and before the CTA exits (a bulk
// copy still landing in shared memory of a finished CTA is not allowed), so
// each kernel's ring spans exactly the planes it reads.
template <int S>
struct Ring {
  unsigned char* base;
  uint64_t* bars;
  int stage_bytes, p0, p1;
  __device__ unsigned char* at(int p) const { return base + ((p - p0) % S) * stage_bytes; }
  __device__ uint64_t* bar(int p) const { return &bars[(p - p0) % S]; }
  __device__ uint32_t parity(int p) const { return ((p - p0) / S) & 1; }
  __device__ bool wait(int p) const { return mbar_wait(bar(p), parity(p), kWaitCycles); }
};

// Common CTA prologue: barrier setup.  Returns the ring.
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
__device__ void ring_drain(const Ring<S>& r, unsigned* err) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    atomicOr(err, ERR_TIMEOUT);
    for (int p = r.p1; p >= r.p0 && p > r.p1 - S; --p) r.wait(p);
  }
}

__device__ __forceinline__ bool tile_in_slab(int lo, int hi_incl, int n, int P) {
  return lo < P || hi_incl >= n - P;
}


// Per-row state of a thread: a thread handles rows ty + r * (TY / RPT),
// r = 0 .. RPT-1, of its 32 x TY tile.
#define ROWS_SETUP()                                                                  \
  constexpr int TYT = TY / RPT;                                                        \
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;                    \
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;                                \
  const int x = x0 + tx;                                                               \
  const int k0 = blockIdx.z * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);

// =================================================== forward H half-step ===
template <int TY, int S>
struct FH {
  typedef SL<TY> L;
  static constexpr int E = 0;                                   // E halo, 3 comps
  static constexpr int H = L::r128(3 * L::HP * 4);              // H own, 3 comps
  static constexpr int PX = H + L::r128(3 * L::OP * 4);         // psi own 2 comps, x/y/z
  static constexpr int PY = PX + L::r128(2 * L::OP * 4);
  static constexpr int PZ = PY + L::r128(2 * L::OP * 4);
  static constexpr int STAGE = PZ + L::r128(2 * L::OP * 4);
  static int smem() { return S * STAGE + 8 * S; }
};

template <int TY, int RPT, int S>
__global__ void __launch_bounds__(32 * TY / RPT) k_sfwd_h(const __grid_constant__ SplitMaps m,
                                                         StepArgs a) {
  typedef SL<TY> L;
  typedef FH<TY, S> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  ROWS_SETUP();
  const bool txs = tile_in_slab(x0, min(x0 + 31, g.nx - 1), g.nx, g.P);
  const bool tys = tile_in_slab(y0, min(y0 + TY - 1, g.ny - 1), g.ny, g.P);
  // planes k0 .. k1 (E at k+1 for the last plane), each waited before reuse
  Ring<S> R = ring_setup<S>(dsm, Y::STAGE, k0, k1);
  auto issue = [&](int p) {
    unsigned char* st = R.at(p);
    uint64_t* bar = R.bar(p);
    const bool body = p >= k0 && p < k1;
    const bool zs = body && in_slab(p, g.nz, g.P);
    uint32_t tx_bytes = 3 * L::HP * 4 + (body ? 3 * L::OP * 4 : 0) +
                        (body && txs ? 2 * L::OP * 4 : 0) + (body && tys ? 2 * L::OP * 4 : 0) +
                        (zs ? 2 * L::OP * 4 : 0);
    mbar_expect_tx(bar, tx_bytes);
    tma_load_4d(st + Y::E, &m.Fh, bar, x0 - 4, y0 - 1, p, 0);
    if (body) tma_load_4d(st + Y::H, &m.Fo, bar, x0, y0, p, 3);
    if (body && txs) tma_load_4d(st + Y::PX, &m.Po, bar, x0, y0, p, 0);
    if (body && tys) tma_load_4d(st + Y::PY, &m.Po, bar, x0, y0, p, 4);
    if (zs) tma_load_4d(st + Y::PZ, &m.Po, bar, x0, y0, p, 8);
    const int pf = p + S;   // warm L2 for the plane this stage will hold next
    if (pf <= R.p1 && pf < g.nz) {
      tma_prefetch_l2_4d(&m.Fh, x0 - 4, y0 - 1, pf, 0);
      if (pf < k1) tma_prefetch_l2_4d(&m.Fo, x0, y0, pf, 3);
    }
  };
  if (tid == 0)
    for (int p = R.p0; p <= R.p1 && p < R.p0 + S; ++p) issue(p);
  const bool sx = x < g.nx && in_slab(x, g.nx, g.P);
  float bx = 0.f, ax = 0.f, kx = 1.f;
  if (sx) { bx = prof(g, 0, PR_BH, x); ax = prof(g, 0, PR_AH, x); kx = prof(g, 0, PR_KH, x); }
  bool valid[RPT], sy[RPT];
  float by[RPT], ay[RPT], ky[RPT];
  long long q[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int y = y0 + ty + r * TYT;
    valid[r] = x < g.nx && y < g.ny;
    sy[r] = valid[r] && in_slab(y, g.ny, g.P);
    by[r] = sy[r] ? prof(g, 1, PR_BH, y) : 0.f;
    ay[r] = sy[r] ? prof(g, 1, PR_AH, y) : 0.f;
    ky[r] = sy[r] ? prof(g, 1, PR_KH, y) : 1.f;
    q[r] = (long long)k0 * g.plane + (long long)y * g.px + x;
  }
  float* F = a.F;
  float* psi = a.psiA;
  const long long nc = g.nc;
  bool ok = true;
  for (int k = k0; k < k1; ++k) {
    if (!R.wait(k) || !R.wait(k + 1)) ok = false;
    if (!__syncthreads_and(ok)) { ring_drain<S>(R, a.err); return; }
    const float* Ec = reinterpret_cast<const float*>(R.at(k) + Y::E);
    const float* En = reinterpret_cast<const float*>(R.at(k + 1) + Y::E);
    const float* Ho = reinterpret_cast<const float*>(R.at(k) + Y::H);
    const bool sz = in_slab(k, g.nz, g.P);
    float bz = 0.f, az = 0.f, kz = 1.f;
    if (sz) { bz = prof(g, 2, PR_BH, k); az = prof(g, 2, PR_AH, k); kz = prof(g, 2, PR_KH, k); }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (!valid[r]) continue;
      const int ty_r = ty + r * TYT;
      const int hi = (ty_r + 1) * L::HW + tx + 4;   // own cell in a halo box
      const int oi = ty_r * L::OW + tx;             // own cell in an own box
      const long long qq = q[r];
      const float ex = Ec[hi], ey = Ec[L::HP + hi], ez = Ec[2 * L::HP + hi];
      const float d0 = Ec[2 * L::HP + hi + L::HW] - ez;   // dEz/dy
      const float d1 = En[L::HP + hi] - ey;               // dEy/dz
      const float d2 = En[hi] - ex;                       // dEx/dz
      const float d3 = Ec[2 * L::HP + hi + 1] - ez;       // dEz/dx
      const float d4 = Ec[L::HP + hi + 1] - ey;           // dEy/dx
      const float d5 = Ec[hi + L::HW] - ex;               // dEx/dy
      float cx, cy, cz;
      if (!(sx || sy[r] || sz)) {
        cx = d0 - d1;
        cy = d2 - d3;
        cz = d4 - d5;
      } else {
        float t0 = d0, t1 = d1, t2 = d2, t3 = d3, t4 = d4, t5 = d5;
        if (sx) {
          const float* P = reinterpret_cast<const float*>(R.at(k) + Y::PX);
          t3 = cpml_s(d3, P[oi], psi, 0 * nc + qq, bx, ax, kx);
          t4 = cpml_s(d4, P[L::OP + oi], psi, 1 * nc + qq, bx, ax, kx);
        }
        if (sy[r]) {
          const float* P = reinterpret_cast<const float*>(R.at(k) + Y::PY);
          t0 = cpml_s(d0, P[oi], psi, 4 * nc + qq, by[r], ay[r], ky[r]);
          t5 = cpml_s(d5, P[L::OP + oi], psi, 5 * nc + qq, by[r], ay[r], ky[r]);
        }
        if (sz) {
          const float* P = reinterpret_cast<const float*>(R.at(k) + Y::PZ);
          t1 = cpml_s(d1, P[oi], psi, 8 * nc + qq, bz, az, kz);
          t2 = cpml_s(d2, P[L::OP + oi], psi, 9 * nc + qq, bz, az, kz);
        }
        cx = t0 - t1;
        cy = t2 - t3;
        cz = t4 - t5;
      }
      F[3 * nc + qq] = __fsub_rn(Ho[oi], __fmul_rn(g.S, cx));
      F[4 * nc + qq] = __fsub_rn(Ho[L::OP + oi], __fmul_rn(g.S, cy));
      F[5 * nc + qq] = __fsub_rn(Ho[2 * L::OP + oi], __fmul_rn(g.S, cz));
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) q[r] += g.plane;
    __syncthreads();
    if (tid == 0 && k + S <= R.p1) issue(k + S);   // plane k is no longer read
  }
}

// =================================================== forward E half-step ===
template <int TY, int S>
struct FE {
  typedef SL<TY> L;
  static constexpr int H = 0;                                   // H halo, 3 comps
  static constexpr int E = L::r128(3 * L::HP * 4);              // E own
  static constexpr int CB = E + L::r128(3 * L::OP * 4);         // cb own
  static constexpr int PX = CB + L::r128(L::OP * 4);
  static constexpr int PY = PX + L::r128(2 * L::OP * 4);
  static constexpr int PZ = PY + L::r128(2 * L::OP * 4);
  static constexpr int STAGE = PZ + L::r128(2 * L::OP * 4);
  static int smem() { return S * STAGE + 8 * S + 256; }
};

template <int TY, int RPT, int S>
__global__ void __launch_bounds__(32 * TY / RPT) k_sfwd_e(const __grid_constant__ SplitMaps m,
                                                         StepArgs a) {
  typedef SL<TY> L;
  typedef FE<TY, S> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  ROWS_SETUP();
  const bool txs = tile_in_slab(x0, min(x0 + 31, g.nx - 1), g.nx, g.P);
  const bool tys = tile_in_slab(y0, min(y0 + TY - 1, g.ny - 1), g.ny, g.P);
  // planes k0-1 .. k1-1 (Ht at k-1 for the first plane), each waited before reuse
  Ring<S> R = ring_setup<S>(dsm, Y::STAGE, k0 - 1, k1 - 1);
  double* red = reinterpret_cast<double*>(dsm + S * Y::STAGE + 8 * S + 64);
  auto issue = [&](int p) {
    unsigned char* st = R.at(p);
    uint64_t* bar = R.bar(p);
    const bool body = p >= k0 && p < k1;
    const bool zs = body && in_slab(p, g.nz, g.P);
    uint32_t tx_bytes = 3 * L::HP * 4 + (body ? 4 * L::OP * 4 : 0) +
                        (body && txs ? 2 * L::OP * 4 : 0) + (body && tys ? 2 * L::OP * 4 : 0) +
                        (zs ? 2 * L::OP * 4 : 0);
    mbar_expect_tx(bar, tx_bytes);
    tma_load_4d(st + Y::H, &m.Fh, bar, x0 - 4, y0 - 1, p, 3);
    if (body) {
      tma_load_4d(st + Y::E, &m.Fo, bar, x0, y0, p, 0);
      tma_load_4d(st + Y::CB, &m.cbo, bar, x0, y0, p, 0);
    }
    if (body && txs) tma_load_4d(st + Y::PX, &m.Po, bar, x0, y0, p, 2);
    if (body && tys) tma_load_4d(st + Y::PY, &m.Po, bar, x0, y0, p, 6);
    if (zs) tma_load_4d(st + Y::PZ, &m.Po, bar, x0, y0, p, 10);
    const int pf = p + S;
    if (pf <= R.p1 && pf >= 0 && pf < g.nz) {
      tma_prefetch_l2_4d(&m.Fh, x0 - 4, y0 - 1, pf, 3);
      tma_prefetch_l2_4d(&m.Fo, x0, y0, pf, 0);
      tma_prefetch_l2_4d(&m.cbo, x0, y0, pf, 0);
    }
  };
  if (tid == 0)
    for (int p = R.p0; p <= R.p1 && p < R.p0 + S; ++p) issue(p);
  const bool sx = x < g.nx && in_slab(x, g.nx, g.P);
  float bx = 0.f, ax = 0.f, kx = 1.f;
  if (sx) { bx = prof(g, 0, PR_BE, x); ax = prof(g, 0, PR_AE, x); kx = prof(g, 0, PR_KE, x); }
  bool valid[RPT], sy[RPT];
  float by[RPT], ay[RPT], ky[RPT];
  long long q[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int y = y0 + ty + r * TYT;
    valid[r] = x < g.nx && y < g.ny;
    sy[r] = valid[r] && in_slab(y, g.ny, g.P);
    by[r] = sy[r] ? prof(g, 1, PR_BE, y) : 0.f;
    ay[r] = sy[r] ? prof(g, 1, PR_AE, y) : 0.f;
    ky[r] = sy[r] ? prof(g, 1, PR_KE, y) : 1.f;
    q[r] = (long long)k0 * g.plane + (long long)y * g.px + x;
  }
  // source and detector planes this thread's columns can cross
  const bool src_on = a.src.kind != 0;
  const bool det_on = a.det.kind != 0;
  float* F = a.F;
  float* psi = a.psiA;
  const long long nc = g.nc;
  double lsum = 0.0;
  bool ok = true;
  for (int k = k0; k < k1; ++k) {
    if (!R.wait(k - 1) || !R.wait(k)) ok = false;
    if (!__syncthreads_and(ok)) { ring_drain<S>(R, a.err); return; }
    const float* Hc = reinterpret_cast<const float*>(R.at(k) + Y::H);
    const float* Hm = reinterpret_cast<const float*>(R.at(k - 1) + Y::H);
    const float* Eo = reinterpret_cast<const float*>(R.at(k) + Y::E);
    const float* CB = reinterpret_cast<const float*>(R.at(k) + Y::CB);
    const bool sz = in_slab(k, g.nz, g.P);
    float bz = 0.f, az = 0.f, kz = 1.f;
    if (sz) { bz = prof(g, 2, PR_BE, k); az = prof(g, 2, PR_AE, k); kz = prof(g, 2, PR_KE, k); }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (!valid[r]) continue;
      const int ty_r = ty + r * TYT;
      const int y = y0 + ty_r;
      const int hi = (ty_r + 1) * L::HW + tx + 4;
      const int oi = ty_r * L::OW + tx;
      const long long qq = q[r];
      const float hx = Hc[hi], hy = Hc[L::HP + hi], hz = Hc[2 * L::HP + hi];
      const float d6 = hz - Hc[2 * L::HP + hi - L::HW];   // dHz/dy
      const float d7 = hy - Hm[L::HP + hi];               // dHy/dz
      const float d8 = hx - Hm[hi];                       // dHx/dz
      const float d9 = hz - Hc[2 * L::HP + hi - 1];       // dHz/dx
      const float d10 = hy - Hc[L::HP + hi - 1];          // dHy/dx
      const float d11 = hx - Hc[hi - L::HW];              // dHx/dy
      float c0, c1, c2;
      if (!(sx || sy[r] || sz)) {
        c0 = d6 - d7;
        c1 = d8 - d9;
        c2 = d10 - d11;
      } else {
        float t6 = d6, t7 = d7, t8 = d8, t9 = d9, t10 = d10, t11 = d11;
        if (sx) {
          const float* P = reinterpret_cast<const float*>(R.at(k) + Y::PX);
          t9 = cpml_s(d9, P[oi], psi, 2 * nc + qq, bx, ax, kx);
          t10 = cpml_s(d10, P[L::OP + oi], psi, 3 * nc + qq, bx, ax, kx);
        }
        if (sy[r]) {
          const float* P = reinterpret_cast<const float*>(R.at(k) + Y::PY);
          t6 = cpml_s(d6, P[oi], psi, 6 * nc + qq, by[r], ay[r], ky[r]);
          t11 = cpml_s(d11, P[L::OP + oi], psi, 7 * nc + qq, by[r], ay[r], ky[r]);
        }
        if (sz) {
          const float* P = reinterpret_cast<const float*>(R.at(k) + Y::PZ);
          t7 = cpml_s(d7, P[oi], psi, 10 * nc + qq, bz, az, kz);
          t8 = cpml_s(d8, P[L::OP + oi], psi, 11 * nc + qq, bz, az, kz);
        }
        c0 = t6 - t7;
        c1 = t8 - t9;
        c2 = t10 - t11;
      }
      if (src_on) {
        const float w = src_wt(a.src, x, y, k);
        if (w != 0.f) {
          const float wj = __fmul_rn(w, a.jn);
          if (a.src.comp == 0) c0 = __fsub_rn(c0, wj);
          else if (a.src.comp == 1) c1 = __fsub_rn(c1, wj);
          else c2 = __fsub_rn(c2, wj);
        }
      }
      const float cbv = CB[oi];
      const float ex = __fadd_rn(Eo[oi], __fmul_rn(cbv, c0));
      const float ey = __fadd_rn(Eo[L::OP + oi], __fmul_rn(cbv, c1));
      const float ez = __fadd_rn(Eo[2 * L::OP + oi], __fmul_rn(cbv, c2));
      F[qq] = ex;
      F[nc + qq] = ey;
      F[2 * nc + qq] = ez;
      int u, v;
      if (det_on && on_plane(a.det.axis, a.det.index, a.det.u0, a.det.u1, a.det.v0, a.det.v1,
                             x, y, k, &u, &v)) {
        if (a.det.kind == 1) {
          lsum += (double)ex * ex + (double)ey * ey + (double)ez * ez;
        } else {
          const int ax_ = a.det.axis;
          const float Eb = ax_ == 0 ? ey : (ax_ == 1 ? ez : ex);
          const float Ec2 = ax_ == 0 ? ez : (ax_ == 1 ? ex : ey);
          const float Hb = ax_ == 0 ? hy : (ax_ == 1 ? hz : hx);
          const float Hc2 = ax_ == 0 ? hz : (ax_ == 1 ? hx : hy);
          lsum += (double)Eb * Hc2 - (double)Ec2 * Hb;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) q[r] += g.plane;
    __syncthreads();
    if (tid == 0 && k - 1 + S <= R.p1) issue(k - 1 + S);
  }
  if (det_on) {
    double v = lsum;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int wv = 0; wv < TYT; ++wv) t += red[wv];
      if (t != 0.0) atomicAdd(a.obj, t);
    }
  }
}

// ======================================== reverse E phase (+ adjoint H) ===
template <int TY, int S>
struct RE {
  typedef SL<TY> L;
  static constexpr int H = 0;                                   // H halo
  static constexpr int E = L::r128(3 * L::HP * 4);              // E own
  static constexpr int CB = E + L::r128(3 * L::OP * 4);         // cb halo
  static constexpr int LE = CB + L::r128(L::HP * 4);            // lam_E halo
  static constexpr int LH = LE + L::r128(3 * L::HP * 4);        // lam_H own
  static constexpr int PX = LH + L::r128(3 * L::OP * 4);        // lam_psi_E halo, 2 comps
  static constexpr int PY = PX + L::r128(2 * L::HP * 4);
  static constexpr int PZ = PY + L::r128(2 * L::HP * 4);
  static constexpr int STAGE = PZ + L::r128(2 * L::HP * 4);
  static int smem() { return S * STAGE + 8 * S; }
};

template <int TY, int RPT, int S>
__global__ void __launch_bounds__(32 * TY / RPT) k_srev_e(const __grid_constant__ SplitMaps m,
                                                         StepArgs a) {
  typedef SL<TY> L;
  typedef RE<TY, S> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  ROWS_SETUP();
  // slab flags include the +1 neighbours the adjoint reads
  const bool txs = tile_in_slab(x0, min(x0 + 32, g.nx - 1), g.nx, g.P);
  const bool tys = tile_in_slab(y0, min(y0 + TY, g.ny - 1), g.ny, g.P);
  const bool tint = x0 + 31 >= g.P && x0 < g.nx - g.P && y0 + TY - 1 >= g.P && y0 < g.ny - g.P;
  Ring<S> R = ring_setup<S>(dsm, Y::STAGE, k0 - 1, k1);
  auto issue = [&](int p) {
    unsigned char* st = R.at(p);
    uint64_t* bar = R.bar(p);
    const bool body = p >= k0 && p < k1;
    const bool zs = p >= k0 && in_slab(p, g.nz, g.P) && p < g.nz;
    uint32_t tx_bytes = 3 * L::HP * 4 + L::HP * 4 + 3 * L::HP * 4 +
                        (body ? 6 * L::OP * 4 : 0) + (body && txs ? 2 * L::HP * 4 : 0) +
                        (body && tys ? 2 * L::HP * 4 : 0) + (zs ? 2 * L::HP * 4 : 0);
    mbar_expect_tx(bar, tx_bytes);
    tma_load_4d(st + Y::H, &m.Fh, bar, x0 - 4, y0 - 1, p, 3);
    tma_load_4d(st + Y::CB, &m.cbh, bar, x0 - 4, y0 - 1, p, 0);
    tma_load_4d(st + Y::LE, &m.Lh, bar, x0 - 4, y0 - 1, p, 0);
    if (body) {
      tma_load_4d(st + Y::E, &m.Fo, bar, x0, y0, p, 0);
      tma_load_4d(st + Y::LH, &m.Lo, bar, x0, y0, p, 3);
    }
    const int pf = p + S;
    if (pf <= R.p1 && pf >= 0 && pf < g.nz) {
      tma_prefetch_l2_4d(&m.Fh, x0 - 4, y0 - 1, pf, 3);
      tma_prefetch_l2_4d(&m.cbh, x0 - 4, y0 - 1, pf, 0);
      tma_prefetch_l2_4d(&m.Lh, x0 - 4, y0 - 1, pf, 0);
      if (pf < k1) {
        tma_prefetch_l2_4d(&m.Fo, x0, y0, pf, 0);
        tma_prefetch_l2_4d(&m.Lo, x0, y0, pf, 3);
      }
    }
    if (body && txs) tma_load_4d(st + Y::PX, &m.Ph, bar, x0 - 4, y0 - 1, p, 2);
    if (body && tys) tma_load_4d(st + Y::PY, &m.Ph, bar, x0 - 4, y0 - 1, p, 6);
    if (zs) tma_load_4d(st + Y::PZ, &m.Ph, bar, x0 - 4, y0 - 1, p, 10);
  };
  if (tid == 0)
    for (int p = R.p0; p <= R.p1 && p < R.p0 + S; ++p) issue(p);
  const bool xv = x < g.nx;
  const bool sx = xv && in_slab(x, g.nx, g.P), sx1 = x + 1 < g.nx && in_slab(x + 1, g.nx, g.P);
  float bx = 0.f, ax = 0.f, kx = 1.f, bx1 = 0.f, ax1 = 0.f, kx1 = 1.f;
  if (sx) { bx = prof(g, 0, PR_BE, x); ax = prof(g, 0, PR_AE, x); kx = prof(g, 0, PR_KE, x); }
  if (sx1) { bx1 = prof(g, 0, PR_BE, x + 1); ax1 = prof(g, 0, PR_AE, x + 1); kx1 = prof(g, 0, PR_KE, x + 1); }
  const bool xin = x >= g.P && x < g.nx - g.P;
  const bool dx_in = x >= a.dlo[0] && x < a.dhi[0];
  const int dX = a.dhi[0] - a.dlo[0], dY = a.dhi[1] - a.dlo[1];
  bool valid[RPT];
  long long q[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int y = y0 + ty + r * TYT;
    valid[r] = xv && y < g.ny;
    q[r] = (long long)k0 * g.plane + (long long)y * g.px + x;
  }
  float* F = a.F;
  float* LL = a.L;
  float* lpB = a.psiB;
  const long long nc = g.nc;
  const bool src_on = a.src.kind != 0;
  bool ok = true;
  for (int k = k0; k < k1; ++k) {
    if (!R.wait(k - 1) || !R.wait(k) || !R.wait(k + 1)) ok = false;
    if (!__syncthreads_and(ok)) { ring_drain<S>(R, a.err); return; }
    const unsigned char* sc = R.at(k);
    const unsigned char* sn = R.at(k + 1);
    const float* LEc = reinterpret_cast<const float*>(sc + Y::LE);
    const float* CBc = reinterpret_cast<const float*>(sc + Y::CB);
    const float* LEn = reinterpret_cast<const float*>(sn + Y::LE);
    const float* CBn = reinterpret_cast<const float*>(sn + Y::CB);
    const float* Hc = reinterpret_cast<const float*>(sc + Y::H);
    const float* Hm = reinterpret_cast<const float*>(R.at(k - 1) + Y::H);
    const float* Eo = reinterpret_cast<const float*>(sc + Y::E);
    const float* LHo = reinterpret_cast<const float*>(sc + Y::LH);
    const bool kin = k >= g.P && k < g.nz - g.P;
    const bool dk_in = k >= a.dlo[2] && k < a.dhi[2];
    const bool sz = in_slab(k, g.nz, g.P), sz1 = k + 1 < g.nz && in_slab(k + 1, g.nz, g.P);
    const bool zlast = k + 1 >= g.nz;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (!valid[r]) continue;
      const int ty_r = ty + r * TYT;
      const int y = y0 + ty_r;
      const int hi = (ty_r + 1) * L::HW + tx + 4;
      const int oi = ty_r * L::OW + tx;
      const long long qq = q[r];
      const float cbv = CBc[hi];
      const float lex = LEc[hi], ley = LEc[L::HP + hi], lez = LEc[2 * L::HP + hi];
      // primal inverse E update on the interior, dL/dcb on the design box
      if (tint && xin && kin && y >= g.P && y < g.ny - g.P) {
        const float hx = Hc[hi], hy = Hc[L::HP + hi], hz = Hc[2 * L::HP + hi];
        const float d6 = hz - Hc[2 * L::HP + hi - L::HW], d7 = hy - Hm[L::HP + hi];
        const float d8 = hx - Hm[hi], d9 = hz - Hc[2 * L::HP + hi - 1];
        const float d10 = hy - Hc[L::HP + hi - 1], d11 = hx - Hc[hi - L::HW];
        float c0 = d6 - d7, c1 = d8 - d9, c2 = d10 - d11;
        if (src_on) {
          const float w = src_wt(a.src, x, y, k);
          if (w != 0.f) {
            const float wj = __fmul_rn(w, a.jn);
            if (a.src.comp == 0) c0 = __fsub_rn(c0, wj);
            else if (a.src.comp == 1) c1 = __fsub_rn(c1, wj);
            else c2 = __fsub_rn(c2, wj);
          }
        }
        F[qq] = __fsub_rn(Eo[oi], __fmul_rn(cbv, c0));
        F[nc + qq] = __fsub_rn(Eo[L::OP + oi], __fmul_rn(cbv, c1));
        F[2 * nc + qq] = __fsub_rn(Eo[2 * L::OP + oi], __fmul_rn(cbv, c2));
        if (dx_in && dk_in && y >= a.dlo[1] && y < a.dhi[1]) {
          const float s = lex * c0 + ley * c1 + lez * c2;
          const long long qd = ((long long)(k - a.dlo[2]) * dY + (y - a.dlo[1])) * dX + (x - a.dlo[0]);
          a.gacc[qd] += (double)s;
        }
      }
      // adjoint of the E half-step: lam_H += D'^T lam_delta'
      const float wx = cbv * lex, wy = cbv * ley, wz = cbv * lez;
      float o6 = wx, o11 = -wz, o7 = -wx, o8 = wy, o9 = -wy, o10 = wz;
      float n6, n11, n7, n8, n9, n10;
      {  // +y neighbour (terms t6: Ex,y,+ and t11: Ez,y,-)
        const int rr = hi + L::HW;
        const float c2 = CBc[rr];
        n6 = c2 * LEc[rr];
        n11 = -c2 * LEc[2 * L::HP + rr];
      }
      {  // +x neighbour (t9: Ey,x,- and t10: Ez,x,+)
        const int rr = hi + 1;
        const float c2 = CBc[rr];
        n9 = -c2 * LEc[L::HP + rr];
        n10 = c2 * LEc[2 * L::HP + rr];
      }
      {  // +z neighbour (t7: Ex,z,- and t8: Ey,z,+)
        const float c2 = CBn[hi];
        n7 = -c2 * LEn[hi];
        n8 = c2 * LEn[L::HP + hi];
      }
      if (y + 1 >= g.ny) { n6 = 0.f; n11 = 0.f; }
      if (x + 1 >= g.nx) { n9 = 0.f; n10 = 0.f; }
      if (zlast) { n7 = 0.f; n8 = 0.f; }
      const bool sy = in_slab(y, g.ny, g.P), sy1 = y + 1 < g.ny && in_slab(y + 1, g.ny, g.P);
      if (sy || sy1) {
        const float* P = reinterpret_cast<const float*>(sc + Y::PY);
        if (sy) {
          const float b = prof(g, 1, PR_BE, y), aa = prof(g, 1, PR_AE, y), kv = prof(g, 1, PR_KE, y);
          o6 = adj_s(o6, P[hi], lpB, 6 * nc + qq, true, b, aa, kv);
          o11 = adj_s(o11, P[L::HP + hi], lpB, 7 * nc + qq, true, b, aa, kv);
        }
        if (sy1) {
          const float b1 = prof(g, 1, PR_BE, y + 1), a1 = prof(g, 1, PR_AE, y + 1),
                      k1v = prof(g, 1, PR_KE, y + 1);
          n6 = adj_s(n6, P[hi + L::HW], lpB, 0, false, b1, a1, k1v);
          n11 = adj_s(n11, P[L::HP + hi + L::HW], lpB, 0, false, b1, a1, k1v);
        }
      }
      if (sx || sx1) {
        const float* P = reinterpret_cast<const float*>(sc + Y::PX);
        if (sx) {
          o9 = adj_s(o9, P[hi], lpB, 2 * nc + qq, true, bx, ax, kx);
          o10 = adj_s(o10, P[L::HP + hi], lpB, 3 * nc + qq, true, bx, ax, kx);
        }
        if (sx1) {
          n9 = adj_s(n9, P[hi + 1], lpB, 0, false, bx1, ax1, kx1);
          n10 = adj_s(n10, P[L::HP + hi + 1], lpB, 0, false, bx1, ax1, kx1);
        }
      }
      if (sz) {
        const float* P = reinterpret_cast<const float*>(sc + Y::PZ);
        const float b = prof(g, 2, PR_BE, k), aa = prof(g, 2, PR_AE, k), kv = prof(g, 2, PR_KE, k);
        o7 = adj_s(o7, P[hi], lpB, 10 * nc + qq, true, b, aa, kv);
        o8 = adj_s(o8, P[L::HP + hi], lpB, 11 * nc + qq, true, b, aa, kv);
      }
      if (sz1) {
        const float* P = reinterpret_cast<const float*>(sn + Y::PZ);
        const float b1 = prof(g, 2, PR_BE, k + 1), a1 = prof(g, 2, PR_AE, k + 1),
                    k1v = prof(g, 2, PR_KE, k + 1);
        n7 = adj_s(n7, P[hi], lpB, 0, false, b1, a1, k1v);
        n8 = adj_s(n8, P[L::HP + hi], lpB, 0, false, b1, a1, k1v);
      }
      LL[3 * nc + qq] = LHo[oi] + ((o8 - n8) + (o11 - n11));
      LL[4 * nc + qq] = LHo[L::OP + oi] + ((o7 - n7) + (o10 - n10));
      LL[5 * nc + qq] = LHo[2 * L::OP + oi] + ((o6 - n6) + (o9 - n9));
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) q[r] += g.plane;
    __syncthreads();
    if (tid == 0 && k - 1 + S <= R.p1) issue(k - 1 + S);
  }
}

// ======================================== reverse H phase (+ adjoint E) ===
template <int TY, int S>
struct RH {
  typedef SL<TY> L;
  static constexpr int E = 0;                                   // E halo
  static constexpr int H = L::r128(3 * L::HP * 4);              // H own
  static constexpr int LH = H + L::r128(3 * L::OP * 4);         // lam_H halo
  static constexpr int LE = LH + L::r128(3 * L::HP * 4);        // lam_E own
  static constexpr int PX = LE + L::r128(3 * L::OP * 4);        // lam_psi_H halo, 2 comps
  static constexpr int PY = PX + L::r128(2 * L::HP * 4);
  static constexpr int PZ = PY + L::r128(2 * L::HP * 4);
  static constexpr int STAGE = PZ + L::r128(2 * L::HP * 4);
  static int smem() { return S * STAGE + 8 * S; }
};

template <int TY, int RPT, int S>
__global__ void __launch_bounds__(32 * TY / RPT) k_srev_h(const __grid_constant__ SplitMaps m,
                                                         StepArgs a) {
  typedef SL<TY> L;
  typedef RH<TY, S> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  ROWS_SETUP();
  // slab flags include the -1 neighbours the adjoint reads
  const bool txs = tile_in_slab(max(x0 - 1, 0), min(x0 + 31, g.nx - 1), g.nx, g.P);
  const bool tys = tile_in_slab(max(y0 - 1, 0), min(y0 + TY - 1, g.ny - 1), g.ny, g.P);
  const bool tint = x0 + 31 >= g.P && x0 < g.nx - g.P && y0 + TY - 1 >= g.P && y0 < g.ny - g.P;
  Ring<S> R = ring_setup<S>(dsm, Y::STAGE, k0 - 1, k1);
  auto issue = [&](int p) {
    unsigned char* st = R.at(p);
    uint64_t* bar = R.bar(p);
    const bool body = p >= k0 && p < k1;
    const bool zs = p >= 0 && p < k1 && in_slab(p, g.nz, g.P);
    uint32_t tx_bytes = 3 * L::HP * 4 + 3 * L::HP * 4 + (body ? 6 * L::OP * 4 : 0) +
                        (body && txs ? 2 * L::HP * 4 : 0) + (body && tys ? 2 * L::HP * 4 : 0) +
                        (zs ? 2 * L::HP * 4 : 0);
    mbar_expect_tx(bar, tx_bytes);
    tma_load_4d(st + Y::E, &m.Fh, bar, x0 - 4, y0 - 1, p, 0);
    tma_load_4d(st + Y::LH, &m.Lh, bar, x0 - 4, y0 - 1, p, 3);
    if (body) {
      tma_load_4d(st + Y::H, &m.Fo, bar, x0, y0, p, 3);
      tma_load_4d(st + Y::LE, &m.Lo, bar, x0, y0, p, 0);
    }
    const int pf = p + S;
    if (pf <= R.p1 && pf >= 0 && pf < g.nz) {
      tma_prefetch_l2_4d(&m.Fh, x0 - 4, y0 - 1, pf, 0);
      tma_prefetch_l2_4d(&m.Lh, x0 - 4, y0 - 1, pf, 3);
      if (pf < k1) {
        tma_prefetch_l2_4d(&m.Fo, x0, y0, pf, 3);
        tma_prefetch_l2_4d(&m.Lo, x0, y0, pf, 0);
      }
    }
    if (body && txs) tma_load_4d(st + Y::PX, &m.Ph, bar, x0 - 4, y0 - 1, p, 0);
    if (body && tys) tma_load_4d(st + Y::PY, &m.Ph, bar, x0 - 4, y0 - 1, p, 4);
    if (zs) tma_load_4d(st + Y::PZ, &m.Ph, bar, x0 - 4, y0 - 1, p, 8);
  };
  if (tid == 0)
    for (int p = R.p0; p <= R.p1 && p < R.p0 + S; ++p) issue(p);
  const bool xv = x < g.nx;
  const bool sx = xv && in_slab(x, g.nx, g.P), sxm = xv && x > 0 && in_slab(x - 1, g.nx, g.P);
  float bx = 0.f, ax = 0.f, kx = 1.f, bxm = 0.f, axm = 0.f, kxm = 1.f;
  if (sx) { bx = prof(g, 0, PR_BH, x); ax = prof(g, 0, PR_AH, x); kx = prof(g, 0, PR_KH, x); }
  if (sxm) { bxm = prof(g, 0, PR_BH, x - 1); axm = prof(g, 0, PR_AH, x - 1); kxm = prof(g, 0, PR_KH, x - 1); }
  const bool xin = x >= g.P && x < g.nx - g.P;
  bool valid[RPT];
  long long q[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int y = y0 + ty + r * TYT;
    valid[r] = xv && y < g.ny;
    q[r] = (long long)k0 * g.plane + (long long)y * g.px + x;
  }
  const float S_ = g.S;
  float* F = a.F;
  float* LL = a.L;
  float* lpB = a.psiB;
  const long long nc = g.nc;
  bool ok = true;
  for (int k = k0; k < k1; ++k) {
    if (!R.wait(k - 1) || !R.wait(k) || !R.wait(k + 1)) ok = false;
    if (!__syncthreads_and(ok)) { ring_drain<S>(R, a.err); return; }
    const unsigned char* sc = R.at(k);
    const unsigned char* sp = R.at(k - 1);
    const float* Ec = reinterpret_cast<const float*>(sc + Y::E);
    const float* En = reinterpret_cast<const float*>(R.at(k + 1) + Y::E);
    const float* Ho = reinterpret_cast<const float*>(sc + Y::H);
    const float* LHc = reinterpret_cast<const float*>(sc + Y::LH);
    const float* LHp = reinterpret_cast<const float*>(sp + Y::LH);
    const float* LEo = reinterpret_cast<const float*>(sc + Y::LE);
    const bool kin = k >= g.P && k < g.nz - g.P;
    const bool sz = in_slab(k, g.nz, g.P), szm = k > 0 && in_slab(k - 1, g.nz, g.P);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (!valid[r]) continue;
      const int ty_r = ty + r * TYT;
      const int y = y0 + ty_r;
      const int hi = (ty_r + 1) * L::HW + tx + 4;
      const int oi = ty_r * L::OW + tx;
      const long long qq = q[r];
      // primal inverse H update on the interior
      if (tint && xin && kin && y >= g.P && y < g.ny - g.P) {
        const float ex = Ec[hi], ey = Ec[L::HP + hi], ez = Ec[2 * L::HP + hi];
        const float d0 = Ec[2 * L::HP + hi + L::HW] - ez, d1 = En[L::HP + hi] - ey;
        const float d2 = En[hi] - ex, d3 = Ec[2 * L::HP + hi + 1] - ez;
        const float d4 = Ec[L::HP + hi + 1] - ey, d5 = Ec[hi + L::HW] - ex;
        F[3 * nc + qq] = __fadd_rn(Ho[oi], __fmul_rn(S_, d0 - d1));
        F[4 * nc + qq] = __fadd_rn(Ho[L::OP + oi], __fmul_rn(S_, d2 - d3));
        F[5 * nc + qq] = __fadd_rn(Ho[2 * L::OP + oi], __fmul_rn(S_, d4 - d5));
      }
      // adjoint of the H half-step: lam_E += D^T lam_delta, v = -S s lam_H
      const float lhx = LHc[hi], lhy = LHc[L::HP + hi], lhz = LHc[2 * L::HP + hi];
      float o0 = -S_ * lhx, o5 = S_ * lhz, o1 = S_ * lhx, o2 = -S_ * lhy, o3 = S_ * lhy,
            o4 = -S_ * lhz;
      float m0 = -S_ * LHc[hi - L::HW], m5 = S_ * LHc[2 * L::HP + hi - L::HW];   // -y
      float m3 = S_ * LHc[L::HP + hi - 1], m4 = -S_ * LHc[2 * L::HP + hi - 1];   // -x
      float m1 = S_ * LHp[hi], m2 = -S_ * LHp[L::HP + hi];                       // -z
      if (y == 0) { m0 = 0.f; m5 = 0.f; }
      if (x == 0) { m3 = 0.f; m4 = 0.f; }
      if (k == 0) { m1 = 0.f; m2 = 0.f; }
      const bool sy = in_slab(y, g.ny, g.P), sym = y > 0 && in_slab(y - 1, g.ny, g.P);
      if (sy || sym) {
        const float* P = reinterpret_cast<const float*>(sc + Y::PY);
        if (sy) {
          const float b = prof(g, 1, PR_BH, y), aa = prof(g, 1, PR_AH, y), kv = prof(g, 1, PR_KH, y);
          o0 = adj_s(o0, P[hi], lpB, 4 * nc + qq, true, b, aa, kv);
          o5 = adj_s(o5, P[L::HP + hi], lpB, 5 * nc + qq, true, b, aa, kv);
        }
        if (sym) {
          const float b1 = prof(g, 1, PR_BH, y - 1), a1 = prof(g, 1, PR_AH, y - 1),
                      k1v = prof(g, 1, PR_KH, y - 1);
          m0 = adj_s(m0, P[hi - L::HW], lpB, 0, false, b1, a1, k1v);
          m5 = adj_s(m5, P[L::HP + hi - L::HW], lpB, 0, false, b1, a1, k1v);
        }
      }
      if (sx || sxm) {
        const float* P = reinterpret_cast<const float*>(sc + Y::PX);
        if (sx) {
          o3 = adj_s(o3, P[hi], lpB, 0 * nc + qq, true, bx, ax, kx);
          o4 = adj_s(o4, P[L::HP + hi], lpB, 1 * nc + qq, true, bx, ax, kx);
        }
        if (sxm) {
          m3 = adj_s(m3, P[hi - 1], lpB, 0, false, bxm, axm, kxm);
          m4 = adj_s(m4, P[L::HP + hi - 1], lpB, 0, false, bxm, axm, kxm);
        }
      }
      if (sz) {
        const float* P = reinterpret_cast<const float*>(sc + Y::PZ);
        const float b = prof(g, 2, PR_BH, k), aa = prof(g, 2, PR_AH, k), kv = prof(g, 2, PR_KH, k);
        o1 = adj_s(o1, P[hi], lpB, 8 * nc + qq, true, b, aa, kv);
        o2 = adj_s(o2, P[L::HP + hi], lpB, 9 * nc + qq, true, b, aa, kv);
      }
      if (szm) {
        const float* P = reinterpret_cast<const float*>(sp + Y::PZ);
        const float b1 = prof(g, 2, PR_BH, k - 1), a1 = prof(g, 2, PR_AH, k - 1),
                    k1v = prof(g, 2, PR_KH, k - 1);
        m1 = adj_s(m1, P[hi], lpB, 0, false, b1, a1, k1v);
        m2 = adj_s(m2, P[L::HP + hi], lpB, 0, false, b1, a1, k1v);
      }
      LL[qq] = LEo[oi] + ((m2 - o2) + (m5 - o5));
      LL[nc + qq] = LEo[L::OP + oi] + ((m1 - o1) + (m4 - o4));
      LL[2 * nc + qq] = LEo[2 * L::OP + oi] + ((m0 - o0) + (m3 - o3));
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) q[r] += g.plane;
    __syncthreads();
    if (tid == 0 && k - 1 + S <= R.p1) issue(k - 1 + S);
  }
}

// ------------------------------------------------------------ launchers ---
template <class KT>
static cudaError_t set_smem(KT kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int TY, int RPT, int S>
static cudaError_t launch_split_t(int which, const SplitMaps& m, const StepArgs& a,
                                  cudaStream_t s) {
  dim3 grid((a.g.nx + 31) / 32, (a.g.ny + TY - 1) / TY, (a.g.nz + a.zchunk - 1) / a.zchunk);
  dim3 block(32, TY / RPT);
  cudaError_t e = cudaSuccess;
  switch (which) {
    case 0: {
      int sm = FH<TY, S>::smem();
      if ((e = set_smem(k_sfwd_h<TY, RPT, S>, sm))) return e;
      k_sfwd_h<TY, RPT, S><<<grid, block, sm, s>>>(m, a);
      break;
    }
    case 1: {
      int sm = FE<TY, S>::smem();
      if ((e = set_smem(k_sfwd_e<TY, RPT, S>, sm))) return e;
      k_sfwd_e<TY, RPT, S><<<grid, block, sm, s>>>(m, a);
      break;
    }
    case 2: {
      int sm = RE<TY, S>::smem();
      if ((e = set_smem(k_srev_e<TY, RPT, S>, sm))) return e;
      k_srev_e<TY, RPT, S><<<grid, block, sm, s>>>(m, a);
      break;
    }
    case 3: {
      int sm = RH<TY, S>::smem();
      if ((e = set_smem(k_srev_h<TY, RPT, S>, sm))) return e;
      k_srev_h<TY, RPT, S><<<grid, block, sm, s>>>(m, a);
      break;
    }
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// which: 0 forward H, 1 forward E, 2 reverse E phase, 3 reverse H phase.
// a.rows: rows of the tile each thread handles (1 or 2; tile height 1 uses 1).
cudaError_t launch_split_tma(int which, const SplitMaps& m, const StepArgs& a, cudaStream_t s) {
  const bool two = a.rows >= 2;
  switch (a.tile_y) {
    case 1: return launch_split_t<1, 1, 4>(which, m, a, s);
    case 2: return two ? launch_split_t<2, 2, 4>(which, m, a, s) : launch_split_t<2, 1, 4>(which, m, a, s);
    case 4: return two ? launch_split_t<4, 2, 4>(which, m, a, s) : launch_split_t<4, 1, 4>(which, m, a, s);
    case 8: return two ? launch_split_t<8, 2, 4>(which, m, a, s) : launch_split_t<8, 1, 4>(which, m, a, s);
    case 16: return two ? launch_split_t<16, 2, 3>(which, m, a, s) : launch_split_t<16, 1, 3>(which, m, a, s);
  }
  return cudaErrorInvalidValue;
}

// -------------------------------------------------------- tensor maps ---
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn2() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

static cudaError_t enc(CUtensorMap* m, const float* base, const Geo& g, int ncomp, int bx, int by,
                       int bc) {
  auto fn = encode_fn2();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)ncomp};
  cuuint64_t strides[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.plane * 4, (cuuint64_t)g.nc * 4};
  cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, (cuuint32_t)bc};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t encode_split_maps(const float* F, const float* Lm, const float* cb, const float* psiA,
                              const Geo& g, int ty, SplitMaps* m) {
  cudaError_t e;
  if ((e = enc(&m->Fh, F, g, 6, 40, ty + 2, 3))) return e;
  if ((e = enc(&m->Fo, F, g, 6, 32, ty, 3))) return e;
  if ((e = enc(&m->Lh, Lm, g, 6, 40, ty + 2, 3))) return e;
  if ((e = enc(&m->Lo, Lm, g, 6, 32, ty, 3))) return e;
  if ((e = enc(&m->cbh, cb, g, 1, 40, ty + 2, 1))) return e;
  if ((e = enc(&m->cbo, cb, g, 1, 32, ty, 1))) return e;
  if ((e = enc(&m->Ph, psiA, g, 12, 40, ty + 2, 2))) return e;
  return enc(&m->Po, psiA, g, 12, 32, ty, 2);
}

}  // namespace fdtd
