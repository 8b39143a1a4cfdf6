// kernels_lag2.cu -- one-plane-per-iteration half-steps, two x-cells per thread.
//
// The kernels of kernels_lag.cu with each thread owning two neighbouring
// cells of a tile row (x = x0 + 2 tx and x0 + 2 tx + 1).  Own and +-y values
// move between shared memory, registers and global memory 8 bytes at a time,
// the x-neighbour inside the pair is already in a register, and a term that
// the reference formulation evaluates twice is evaluated once:
//   * the adjoint curl terms a cell contributes to its -x neighbour are the
//     terms the neighbour evaluates for itself (inside a pair),
//   * the z-terms that finish lam_H(p-1) (reverse E phase) and the -z terms
//     carried to plane p+1 (reverse H phase) are the own z-terms of plane p.
// Tiles (32 x TY cells), tensor maps, boxes and ring stages are those of
// kernels_lag.cu.  Every cell sees the same sequence of rounded operations,
// with the same association of every sum, so the fields are bit-identical to
// the other kernel variants.  The ring cursor (stage, parity) advances by
// increment instead of a modulo per plane.
#include <cudaTypedefs.h>

#include "lag_common.cuh"

namespace fdtd {

using namespace lag2;

// Batched designs (BM): this CTA's unit (design, tile x, tile y, chunk), and
// the design's own step arguments and tensor maps in global memory; else the
// launch's own.
template <bool BM>
__device__ __forceinline__ int4 batch_unit(const StepArgs& a_) {
  return BM ? a_.bunits[blockIdx.x] : make_int4(0, 0, 0, 0);
}

// Batched designs: the thread that issues the CTA's copies acquires the
// design's tensor maps (in global memory) before its first copy.
template <bool BM>
__device__ __forceinline__ void batch_maps_acquire(const LagMaps& m) {
  if (BM && threadIdx.x == 0 && threadIdx.y == 0) {
    const CUtensorMap* t = &m.Fw;
    for (int i = 0; i < (int)(sizeof(LagMaps) / sizeof(CUtensorMap)); ++i) tensormap_acquire(t + i);
  }
}

// The unit (tile, z chunk) of this CTA of a forward half-step: every unit of
// the grid (chunks offset by zc0), or, in the UM instantiations, the z-only
// (umode 1) or ring (umode 2) units of a fused forward step, whose CPML-free
// units run k_fwd_fused.
template <bool UM, bool BM>
__device__ __forceinline__ void fwd_unit(const StepArgs& a, int4 bu, int* tix, int* tiy, int* cz) {
  if (BM) {
    *tix = bu.y;
    *tiy = bu.z;
    *cz = bu.w;
  } else if (UM && a.umode == 2) {
    ring_unit(a.U, blockIdx.x, tix, tiy, cz);
  } else if (UM) {
    *tix = blockIdx.x + a.U.ix0;
    *tiy = blockIdx.y + a.U.iy0;
    *cz = zonly_chunk(a.U, blockIdx.z);
  } else {
    *tix = blockIdx.x;
    *tiy = blockIdx.y;
    *cz = blockIdx.z + a.zc0;
  }
}

// =================================================== forward H half-step ===
// UM: a fused forward step's CPML units (unit decode by a.umode, Ht^{n+1/2}
// written to a.Fn); else every unit, in place.
template <int TY, int S, int TW, bool EX, bool UM, bool BM>
__global__ void __launch_bounds__(TW / 2 * TY, (min_ctas<TY, S, TW>(true)))
k_l2fwd_h(const __grid_constant__ LagMaps m_, StepArgs a_) {
  const int4 bu = batch_unit<BM>(a_);
  const StepArgs& a = BM ? a_.bargs[bu.x] : a_;
  const LagMaps& m = BM ? a_.bmaps[a.bmap] : m_;
  batch_maps_acquire<BM>(m);
  typedef G<TY, TW> B;
  typedef LFH<TY, S, TW> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * (TW / 2) + tx;
  int tix, tiy, cz;
  fwd_unit<UM, BM>(a, bu, &tix, &tiy, &cz);
  const int x0 = tix * TW, y0 = tiy * TY;
  const int x = x0 + 2 * tx, y = y0 + ty;
  const bool v0 = x < g.nx && y < g.ny, v1 = v0 && x + 1 < g.nx;
  const int k0 = cz * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  const bool txs = tile_in_slab(x0, min(x0 + TW - 1, g.nx - 1), g.nx, g.P);
  const bool tys = tile_in_slab(y0, min(y0 + TY - 1, g.ny - 1), g.ny, g.P);
  // plane p < k1 starts Ht(p); plane p > k0 finishes Ht(p-1) (needs E(p))
  uint64_t* bars = ring_init<S>(dsm, Y::STAGE);
  int qx0, qy0;
  psi_box_starts<TW, TY>(a.pl, x0, y0, &qx0, &qy0);
  auto boxes = [&](int p, auto&& f) {
    const bool body = p < k1;
    const bool zs = body && in_slab(p, g.nz, g.P);
    f(Y::E, &m.Fw, x0, y0, p, 0, 3 * B::P * 4);
    if (body) f(Y::H, &m.Fo, x0, y0, p, 3, 3 * B::OP * 4);
    if (body && txs) f(Y::PX, &m.Qxo, qx0, y0, p, 0, 2 * B::OP * 4);
    if (body && tys) f(Y::PY, &m.Qyo, x0, qy0, p, 0, 2 * B::OP * 4);
    if (zs) f(Y::PZ, &m.Qzo, x0, y0, psi_map(a.pl.ax[2], p), 0, 2 * B::OP * 4);
  };
  auto issue = [&](int p, unsigned char* st, uint64_t* bar) {
    stage_plane(boxes, p, st, bar, a.prefetch && p + 1 <= k1 && p + 1 < g.nz);
  };
  pdl_sync();
  if (tid == 0)
    for (int i = 0; i < S && k0 + i <= k1; ++i) issue(k0 + i, dsm + i * Y::STAGE, bars + i);
  const bool sx0 = v0 && in_slab(x, g.nx, g.P), sx1 = v1 && in_slab(x + 1, g.nx, g.P);
  const bool sy = v0 && in_slab(y, g.ny, g.P);
  float bx0 = 0.f, ax0 = 0.f, kx0 = 1.f, bx1 = 0.f, ax1 = 0.f, kx1 = 1.f;
  float by = 0.f, ay = 0.f, ky = 1.f;
  if (sx0) { bx0 = prof(g, 0, PR_BH, x); ax0 = prof(g, 0, PR_AH, x); kx0 = prof(g, 0, PR_KH, x); }
  if (sx1) { bx1 = prof(g, 0, PR_BH, x + 1); ax1 = prof(g, 0, PR_AH, x + 1); kx1 = prof(g, 0, PR_KH, x + 1); }
  if (sy) { by = prof(g, 1, PR_BH, y); ay = prof(g, 1, PR_AH, y); ky = prof(g, 1, PR_KH, y); }
  const int hb = ty * B::W + 2 * tx;   // own pair in a hi box
  const int ob = ty * TW + 2 * tx;     // own pair in an own box
  const long long nc = g.nc;
  float* const Hx = (UM ? a.Fn : a.F) + 3 * nc;   // Ht^{n+1/2}: in place, or the other buffer
  float* const Hy = Hx + nc;
  float* const Hz = Hy + nc;
  float* const psi = a.psiA;
  long long q = (long long)k0 * g.plane + (long long)y * g.px + x;   // plane of the carried pair
  // carried state of Ht(p-1), per cell of the pair
  float c_ex[2] = {0.f, 0.f}, c_ey[2] = {0.f, 0.f}, c_t0[2] = {0.f, 0.f}, c_t3[2] = {0.f, 0.f};
  float c_t4[2] = {0.f, 0.f}, c_t5[2] = {0.f, 0.f}, c_hx[2] = {0.f, 0.f}, c_hy[2] = {0.f, 0.f};
  float c_hz[2] = {0.f, 0.f}, c_pz0[2] = {0.f, 0.f}, c_pz1[2] = {0.f, 0.f};
  int stg = 0;
  uint32_t par = 0;
  bool ok = true;
  for (int p = k0; p <= k1; ++p) {
    unsigned char* st = dsm + stg * Y::STAGE;
    if (!mbar_wait(bars + stg, par, kWaitCycles)) ok = false;
    if (!__syncthreads_and(ok)) { ring_abort<S>(bars, stg, par, p, k1, a.err); return; }
    const float* Eb = reinterpret_cast<const float*>(st + Y::E);
    if (v0) {
      const float2 ex2 = ld2(Eb, hb), ey2 = ld2(Eb + B::P, hb);
      const float ex[2] = {ex2.x, ex2.y}, ey[2] = {ey2.x, ey2.y};
      if (p > k0) {  // finish Ht(p-1) with dEy/dz and dEx/dz
        const int k = p - 1;
        float t1[2], t2[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          t1[c] = ey[c] - c_ey[c];
          t2[c] = ex[c] - c_ex[c];
        }
        if (in_slab(k, g.nz, g.P)) {
          const float bz = prof(g, 2, PR_BH, k), az = prof(g, 2, PR_AH, k), kz = prof(g, 2, PR_KH, k);
          float s1[2], s2[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            t1[c] = cpml(t1[c], c_pz0[c], bz, az, kz, &s1[c]);
            t2[c] = cpml(t2[c], c_pz1[c], bz, az, kz, &s2[c]);
          }
          const long long qz = psi_ix<2>(a.pl, 0, x, y, k);
          ST2(psi, qz, s1[0], s1[1], true, v1);
          ST2(psi + a.pl.ax[2].cs, qz, s2[0], s2[1], true, v1);
        }
        float hx[2], hy[2], hz[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float cx = c_t0[c] - t1[c], cy = t2[c] - c_t3[c], cz = c_t4[c] - c_t5[c];
          hx[c] = __fsub_rn(c_hx[c], inc_of<EX>(__fmul_rn(g.S, cx), a));
          hy[c] = __fsub_rn(c_hy[c], inc_of<EX>(__fmul_rn(g.S, cy), a));
          hz[c] = __fsub_rn(c_hz[c], inc_of<EX>(__fmul_rn(g.S, cz), a));
        }
        ST2(Hx, q, hx[0], hx[1], true, v1);
        ST2(Hy, q, hy[0], hy[1], true, v1);
        ST2(Hz, q, hz[0], hz[1], true, v1);
        q += g.plane;
      }
      if (p < k1) {  // start Ht(p): x and y derivatives, their psi updates
        const float2 ez2 = ld2(Eb + 2 * B::P, hb);
        const float2 ezy = ld2(Eb + 2 * B::P, hb + B::W), exy = ld2(Eb, hb + B::W);
        const float ezx = Eb[2 * B::P + hb + 2], eyx = Eb[B::P + hb + 2];
        float t0[2] = {ezy.x - ez2.x, ezy.y - ez2.y};   // dEz/dy
        float t3[2] = {ez2.y - ez2.x, ezx - ez2.y};     // dEz/dx
        float t4[2] = {ey[1] - ey[0], eyx - ey[1]};     // dEy/dx
        float t5[2] = {exy.x - ex[0], exy.y - ex[1]};   // dEx/dy
        if (sx0 || sx1) {
          const float* P = reinterpret_cast<const float*>(st + Y::PX);
          const float2 p0 = ld2(P, ob), p1 = ld2(P + B::OP, ob);
          float s3[2] = {0.f, 0.f}, s4[2] = {0.f, 0.f};
          if (sx0) {
            t3[0] = cpml(t3[0], p0.x, bx0, ax0, kx0, &s3[0]);
            t4[0] = cpml(t4[0], p1.x, bx0, ax0, kx0, &s4[0]);
          }
          if (sx1) {
            t3[1] = cpml(t3[1], p0.y, bx1, ax1, kx1, &s3[1]);
            t4[1] = cpml(t4[1], p1.y, bx1, ax1, kx1, &s4[1]);
          }
          const long long qxx = psi_ix<0>(a.pl, 0, x, y, p);
          ST2(psi, qxx, s3[0], s3[1], sx0, sx1);
          ST2(psi + a.pl.ax[0].cs, qxx, s4[0], s4[1], sx0, sx1);
        }
        if (sy) {
          const float* P = reinterpret_cast<const float*>(st + Y::PY);
          const float2 p0 = ld2(P, ob), p1 = ld2(P + B::OP, ob);
          const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
          float s0[2], s5[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            t0[c] = cpml(t0[c], q0[c], by, ay, ky, &s0[c]);
            t5[c] = cpml(t5[c], q1[c], by, ay, ky, &s5[c]);
          }
          const long long qyy = psi_ix<1>(a.pl, 0, x, y, p);
          ST2(psi, qyy, s0[0], s0[1], true, v1);
          ST2(psi + a.pl.ax[1].cs, qyy, s5[0], s5[1], true, v1);
        }
        const float* Ho = reinterpret_cast<const float*>(st + Y::H);
        const float2 h0 = ld2(Ho, ob), h1 = ld2(Ho + B::OP, ob), h2 = ld2(Ho + 2 * B::OP, ob);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          c_ex[c] = ex[c];
          c_ey[c] = ey[c];
          c_t0[c] = t0[c];
          c_t3[c] = t3[c];
          c_t4[c] = t4[c];
          c_t5[c] = t5[c];
        }
        c_hx[0] = h0.x; c_hx[1] = h0.y;
        c_hy[0] = h1.x; c_hy[1] = h1.y;
        c_hz[0] = h2.x; c_hz[1] = h2.y;
        if (in_slab(p, g.nz, g.P)) {
          const float* P = reinterpret_cast<const float*>(st + Y::PZ);
          const float2 p0 = ld2(P, ob), p1 = ld2(P + B::OP, ob);
          c_pz0[0] = p0.x; c_pz0[1] = p0.y;
          c_pz1[0] = p1.x; c_pz1[1] = p1.y;
        }
      }
    }
    __syncthreads();
    if (tid == 0 && p + S <= k1) issue(p + S, st, bars + stg);
    if (++stg == S) { stg = 0; par ^= 1u; }
  }
}

// =================================================== forward E half-step ===
// UM: as in the H half-step (E^{n+1} written to a.Fn, Ht^{n+1/2} read from
// the buffer the tensor map Fw views).
template <int TY, int S, int TW, bool EX, bool UM, bool BM>
__global__ void __launch_bounds__(TW / 2 * TY, (min_ctas<TY, S, TW>(true)))
k_l2fwd_e(const __grid_constant__ LagMaps m_, StepArgs a_) {
  const int4 bu = batch_unit<BM>(a_);
  const StepArgs& a = BM ? a_.bargs[bu.x] : a_;
  const LagMaps& m = BM ? a_.bmaps[a.bmap] : m_;
  batch_maps_acquire<BM>(m);
  typedef G<TY, TW> B;
  typedef LFE<TY, S, TW> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * (TW / 2) + tx;
  int tix, tiy, cz;
  fwd_unit<UM, BM>(a, bu, &tix, &tiy, &cz);
  const int x0 = tix * TW, y0 = tiy * TY;
  const int x = x0 + 2 * tx, y = y0 + ty;
  const bool v0 = x < g.nx && y < g.ny, v1 = v0 && x + 1 < g.nx;
  const int k0 = cz * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  const bool txs = tile_in_slab(x0, min(x0 + TW - 1, g.nx - 1), g.nx, g.P);
  const bool tys = tile_in_slab(y0, min(y0 + TY - 1, g.ny - 1), g.ny, g.P);
  // plane k0-1 only provides Ht(k0-1) at the own pair
  const int p0_ = k0 - 1, p1_ = k1 - 1;
  uint64_t* bars = ring_init<S>(dsm, Y::STAGE);
  double* red = reinterpret_cast<double*>(dsm + S * Y::STAGE + 8 * S + 64);
  int qx0, qy0;
  psi_box_starts<TW, TY>(a.pl, x0, y0, &qx0, &qy0);
  auto boxes = [&](int p, auto&& f) {
    const bool body = p >= k0;
    const bool zs = body && in_slab(p, g.nz, g.P);
    f(Y::H, &m.Fw, x0 - 4, y0 - 1, p, 3, 3 * B::P * 4);
    if (body) {
      f(Y::E, &m.Fo, x0, y0, p, 0, 3 * B::OP * 4);
      f(Y::CB, &m.cbo, x0, y0, p, 0, B::OP * 4);
    }
    if (body && txs) f(Y::PX, &m.Qxo, qx0, y0, p, 2, 2 * B::OP * 4);
    if (body && tys) f(Y::PY, &m.Qyo, x0, qy0, p, 2, 2 * B::OP * 4);
    if (zs) f(Y::PZ, &m.Qzo, x0, y0, psi_map(a.pl.ax[2], p), 2, 2 * B::OP * 4);
  };
  auto issue = [&](int p, unsigned char* st, uint64_t* bar) {
    stage_plane(boxes, p, st, bar, a.prefetch && p + 1 <= p1_ && p + 1 >= 0 && p + 1 < g.nz);
  };
  pdl_sync();
  if (tid == 0)
    for (int i = 0; i < S && p0_ + i <= p1_; ++i) issue(p0_ + i, dsm + i * Y::STAGE, bars + i);
  const bool sx0 = v0 && in_slab(x, g.nx, g.P), sx1 = v1 && in_slab(x + 1, g.nx, g.P);
  const bool sy = v0 && in_slab(y, g.ny, g.P);
  float bx0 = 0.f, ax0 = 0.f, kx0 = 1.f, bx1 = 0.f, ax1 = 0.f, kx1 = 1.f;
  float by = 0.f, ay = 0.f, ky = 1.f;
  if (sx0) { bx0 = prof(g, 0, PR_BE, x); ax0 = prof(g, 0, PR_AE, x); kx0 = prof(g, 0, PR_KE, x); }
  if (sx1) { bx1 = prof(g, 0, PR_BE, x + 1); ax1 = prof(g, 0, PR_AE, x + 1); kx1 = prof(g, 0, PR_KE, x + 1); }
  if (sy) { by = prof(g, 1, PR_BE, y); ay = prof(g, 1, PR_AE, y); ky = prof(g, 1, PR_KE, y); }
  const int lb = (ty + 1) * B::W + 2 * tx + 4;   // own pair in a lo box
  const int ob = ty * TW + 2 * tx;
  const long long nc = g.nc;
  float* const Ex = UM ? a.Fn : a.F;   // E^{n+1}: in place, or the other buffer
  float* const Ey = Ex + nc;
  float* const Ez = Ey + nc;
  float* const psi = a.psiA;
  long long q = (long long)k0 * g.plane + (long long)y * g.px + x;
  float c_hx[2] = {0.f, 0.f}, c_hy[2] = {0.f, 0.f};   // Ht(p-1) at the own pair
  double lsum = 0.0;
  int stg = 0;
  uint32_t par = 0;
  bool ok = true;
  for (int p = p0_; p <= p1_; ++p) {
    unsigned char* st = dsm + stg * Y::STAGE;
    if (!mbar_wait(bars + stg, par, kWaitCycles)) ok = false;
    if (!__syncthreads_and(ok)) { ring_abort<S>(bars, stg, par, p, p1_, a.err); return; }
    const float* Hb = reinterpret_cast<const float*>(st + Y::H);
    if (v0) {
      const float2 hx2 = ld2(Hb, lb), hy2 = ld2(Hb + B::P, lb), hz2 = ld2(Hb + 2 * B::P, lb);
      const float hx[2] = {hx2.x, hx2.y}, hy[2] = {hy2.x, hy2.y}, hz[2] = {hz2.x, hz2.y};
      if (p >= k0) {
        const int k = p;
        const float2 hzy = ld2(Hb + 2 * B::P, lb - B::W), hxy = ld2(Hb, lb - B::W);
        const float hzx = Hb[2 * B::P + lb - 1], hyx = Hb[B::P + lb - 1];
        const float d6[2] = {hz[0] - hzy.x, hz[1] - hzy.y};      // dHz/dy
        const float d7[2] = {hy[0] - c_hy[0], hy[1] - c_hy[1]};  // dHy/dz
        const float d8[2] = {hx[0] - c_hx[0], hx[1] - c_hx[1]};  // dHx/dz
        const float d9[2] = {hz[0] - hzx, hz[1] - hz[0]};        // dHz/dx
        const float d10[2] = {hy[0] - hyx, hy[1] - hy[0]};       // dHy/dx
        const float d11[2] = {hx[0] - hxy.x, hx[1] - hxy.y};     // dHx/dy
        const bool sz = in_slab(k, g.nz, g.P);
        float c0[2], c1[2], c2[2];
        if (!(sx0 || sx1 || sy || sz)) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            c0[c] = d6[c] - d7[c];
            c1[c] = d8[c] - d9[c];
            c2[c] = d10[c] - d11[c];
          }
        } else {
          float t6[2], t7[2], t8[2], t9[2], t10[2], t11[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            t6[c] = d6[c]; t7[c] = d7[c]; t8[c] = d8[c];
            t9[c] = d9[c]; t10[c] = d10[c]; t11[c] = d11[c];
          }
          if (sx0 || sx1) {
            const float* P = reinterpret_cast<const float*>(st + Y::PX);
            const float2 p0 = ld2(P, ob), p1 = ld2(P + B::OP, ob);
            float s9[2] = {0.f, 0.f}, s10[2] = {0.f, 0.f};
            if (sx0) {
              t9[0] = cpml(d9[0], p0.x, bx0, ax0, kx0, &s9[0]);
              t10[0] = cpml(d10[0], p1.x, bx0, ax0, kx0, &s10[0]);
            }
            if (sx1) {
              t9[1] = cpml(d9[1], p0.y, bx1, ax1, kx1, &s9[1]);
              t10[1] = cpml(d10[1], p1.y, bx1, ax1, kx1, &s10[1]);
            }
            const long long qxx = psi_ix<0>(a.pl, 2, x, y, k);
            ST2(psi, qxx, s9[0], s9[1], sx0, sx1);
            ST2(psi + a.pl.ax[0].cs, qxx, s10[0], s10[1], sx0, sx1);
          }
          if (sy) {
            const float* P = reinterpret_cast<const float*>(st + Y::PY);
            const float2 p0 = ld2(P, ob), p1 = ld2(P + B::OP, ob);
            const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
            float s6[2], s11[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              t6[c] = cpml(d6[c], q0[c], by, ay, ky, &s6[c]);
              t11[c] = cpml(d11[c], q1[c], by, ay, ky, &s11[c]);
            }
            const long long qyy = psi_ix<1>(a.pl, 2, x, y, k);
            ST2(psi, qyy, s6[0], s6[1], true, v1);
            ST2(psi + a.pl.ax[1].cs, qyy, s11[0], s11[1], true, v1);
          }
          if (sz) {
            const float* P = reinterpret_cast<const float*>(st + Y::PZ);
            const float bz = prof(g, 2, PR_BE, k), az = prof(g, 2, PR_AE, k), kz = prof(g, 2, PR_KE, k);
            const float2 p0 = ld2(P, ob), p1 = ld2(P + B::OP, ob);
            const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
            float s7[2], s8[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              t7[c] = cpml(d7[c], q0[c], bz, az, kz, &s7[c]);
              t8[c] = cpml(d8[c], q1[c], bz, az, kz, &s8[c]);
            }
            const long long qz = psi_ix<2>(a.pl, 2, x, y, k);
            ST2(psi, qz, s7[0], s7[1], true, v1);
            ST2(psi + a.pl.ax[2].cs, qz, s8[0], s8[1], true, v1);
          }
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            c0[c] = t6[c] - t7[c];
            c1[c] = t8[c] - t9[c];
            c2[c] = t10[c] - t11[c];
          }
        }
        if (a.src.kind) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const float w = (c == 0 || v1) ? src_wt(a.src, x + c, y, k) : 0.f;
            if (w != 0.f) {
              const float wj = __fmul_rn(w, a.jn);
              if (a.src.comp == 0) c0[c] = __fsub_rn(c0[c], wj);
              else if (a.src.comp == 1) c1[c] = __fsub_rn(c1[c], wj);
              else c2[c] = __fsub_rn(c2[c], wj);
            }
          }
        }
        const float* Eo = reinterpret_cast<const float*>(st + Y::E);
        const float2 cb2 = ld2(reinterpret_cast<const float*>(st + Y::CB), ob);
        const float2 e0 = ld2(Eo, ob), e1 = ld2(Eo + B::OP, ob), e2 = ld2(Eo + 2 * B::OP, ob);
        const float cbv[2] = {cb2.x, cb2.y};
        const float eo0[2] = {e0.x, e0.y}, eo1[2] = {e1.x, e1.y}, eo2[2] = {e2.x, e2.y};
        float ex[2], ey[2], ez[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          ex[c] = __fadd_rn(eo0[c], inc_of<EX>(__fmul_rn(cbv[c], c0[c]), a));
          ey[c] = __fadd_rn(eo1[c], inc_of<EX>(__fmul_rn(cbv[c], c1[c]), a));
          ez[c] = __fadd_rn(eo2[c], inc_of<EX>(__fmul_rn(cbv[c], c2[c]), a));
        }
        ST2(Ex, q, ex[0], ex[1], true, v1);
        ST2(Ey, q, ey[0], ey[1], true, v1);
        ST2(Ez, q, ez[0], ez[1], true, v1);
        if (a.det.kind) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            int u, v;
            if ((c == 0 || v1) && on_plane(a.det.axis, a.det.index, a.det.u0, a.det.u1, a.det.v0,
                                           a.det.v1, x + c, y, k, &u, &v)) {
              if (a.det.kind == 1) {
                lsum += (double)ex[c] * ex[c] + (double)ey[c] * ey[c] + (double)ez[c] * ez[c];
              } else {
                const int ax_ = a.det.axis;
                const float Eb_ = ax_ == 0 ? ey[c] : (ax_ == 1 ? ez[c] : ex[c]);
                const float Ec2 = ax_ == 0 ? ez[c] : (ax_ == 1 ? ex[c] : ey[c]);
                const float Hb2 = ax_ == 0 ? hy[c] : (ax_ == 1 ? hz[c] : hx[c]);
                const float Hc2 = ax_ == 0 ? hz[c] : (ax_ == 1 ? hx[c] : hy[c]);
                lsum += (double)Eb_ * Hc2 - (double)Ec2 * Hb2;
              }
            }
          }
        }
        q += g.plane;
      }
      c_hx[0] = hx[0]; c_hx[1] = hx[1];
      c_hy[0] = hy[0]; c_hy[1] = hy[1];
    }
    __syncthreads();
    if (tid == 0 && p + S <= p1_) issue(p + S, st, bars + stg);
    if (++stg == S) { stg = 0; par ^= 1u; }
  }
  if (a.det.kind) {
    double v = lsum;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int wv = 0; wv < (TW / 2 * TY) / 32; ++wv) t += red[wv];
      if (t != 0.0) atomicAdd(a.obj, t);
    }
  }
}

// ======================================== reverse E phase (+ adjoint H) ===
template <int TY, int S, int TW, bool EX, bool BM>
__global__ void __launch_bounds__(TW / 2 * TY, (min_ctas<TY, S, TW>(false)))
k_l2rev_e(const __grid_constant__ LagMaps m_, StepArgs a_) {
  const int4 bu = batch_unit<BM>(a_);
  const StepArgs& a = BM ? a_.bargs[bu.x] : a_;
  const LagMaps& m = BM ? a_.bmaps[a.bmap] : m_;
  batch_maps_acquire<BM>(m);
  typedef G<TY, TW> B;
  typedef LRE<TY, S, TW> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * (TW / 2) + tx;
  const int x0 = (BM ? bu.y : (int)blockIdx.x) * TW, y0 = (BM ? bu.z : (int)blockIdx.y) * TY;
  const int x = x0 + 2 * tx, y = y0 + ty;
  const bool v0 = x < g.nx && y < g.ny, v1 = v0 && x + 1 < g.nx;
  const int k0 = (BM ? bu.w : (int)blockIdx.z + a.zc0) * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  const bool txs = tile_in_slab(x0, min(x0 + TW, g.nx - 1), g.nx, g.P);
  const bool tys = tile_in_slab(y0, min(y0 + TY, g.ny - 1), g.ny, g.P);
  const bool tint = x0 + TW - 1 >= g.P && x0 < g.nx - g.P && y0 + TY - 1 >= g.P && y0 < g.ny - g.P;
  // plane k0-1: Ht(k0-1) at the own pair; planes k0..k1-1: the step proper,
  // each also finishing lam_H(p-1) with its own z-terms; plane k1 finishes
  // lam_H(k1-1).
  const int p0_ = k0 - 1, p1_ = k1;
  uint64_t* bars = ring_init<S>(dsm, Y::STAGE);
  // primal data only where the primal runs: interior tiles, planes P..nz-P-1
  // (and plane P-1's Ht for the z difference of plane P)
  auto primal_plane = [&](int p) { return tint && p >= g.P && p < g.nz - g.P; };
  int qx0, qy0;
  psi_box_starts<TW, TY>(a.pl, x0, y0, &qx0, &qy0);
  auto boxes = [&](int p, auto&& f) {
    const bool head = p < k0, body = p >= k0 && p < k1, tail = p > k0;
    const bool zs = p >= 0 && p < g.nz && in_slab(p, g.nz, g.P) && (body || tail);
    const bool lam = body || tail;
    const bool hbox = (head || body) && (primal_plane(p) || primal_plane(p + 1));
    const bool ebox = body && primal_plane(p);
    if (hbox) f(Y::H, &m.Fw, x0 - 4, y0 - 1, p, 3, 3 * B::P * 4);
    if (lam) {
      f(Y::CB, &m.cbw, x0, y0, p, 0, B::P * 4);
      f(Y::LE, &m.Lw, x0, y0, p, 0, 3 * B::P * 4);
    }
    if (ebox) f(Y::E, &m.Fo, x0, y0, p, 0, 3 * B::OP * 4);
    if (body) f(Y::LH, &m.Lo, x0, y0, p, 3, 3 * B::OP * 4);
    if (body && txs) f(Y::PX, &m.Qxw, qx0, y0, p, 2, 2 * B::XP * 4);
    if (body && tys) f(Y::PY, &m.Qyw, x0, qy0, p, 2, 2 * B::YP * 4);
    if (zs) f(Y::PZ, &m.Qzo, x0, y0, psi_map(a.pl.ax[2], p), 2, 2 * B::OP * 4);
  };
  auto issue = [&](int p, unsigned char* st, uint64_t* bar) {
    stage_plane(boxes, p, st, bar, a.prefetch && p + 1 <= p1_ && p + 1 >= 0 && p + 1 < g.nz);
  };
  pdl_sync();
  if (tid == 0)
    for (int i = 0; i < S && p0_ + i <= p1_; ++i) issue(p0_ + i, dsm + i * Y::STAGE, bars + i);
  // x profiles at x, x+1 (cell 1, also cell 0's +x neighbour) and x+2
  const bool sx0 = v0 && in_slab(x, g.nx, g.P), sx1 = v1 && in_slab(x + 1, g.nx, g.P);
  const bool sx2 = v1 && x + 2 < g.nx && in_slab(x + 2, g.nx, g.P);
  const bool sy = v0 && in_slab(y, g.ny, g.P), sy1 = v0 && y + 1 < g.ny && in_slab(y + 1, g.ny, g.P);
  float bx0 = 0.f, ax0 = 0.f, kx0 = 1.f, bx1 = 0.f, ax1 = 0.f, kx1 = 1.f, bx2 = 0.f, ax2 = 0.f, kx2 = 1.f;
  float by = 0.f, ay = 0.f, ky = 1.f, by1 = 0.f, ay1 = 0.f, ky1 = 1.f;
  if (sx0) { bx0 = prof(g, 0, PR_BE, x); ax0 = prof(g, 0, PR_AE, x); kx0 = prof(g, 0, PR_KE, x); }
  if (sx1) { bx1 = prof(g, 0, PR_BE, x + 1); ax1 = prof(g, 0, PR_AE, x + 1); kx1 = prof(g, 0, PR_KE, x + 1); }
  if (sx2) { bx2 = prof(g, 0, PR_BE, x + 2); ax2 = prof(g, 0, PR_AE, x + 2); kx2 = prof(g, 0, PR_KE, x + 2); }
  if (sy) { by = prof(g, 1, PR_BE, y); ay = prof(g, 1, PR_AE, y); ky = prof(g, 1, PR_KE, y); }
  if (sy1) { by1 = prof(g, 1, PR_BE, y + 1); ay1 = prof(g, 1, PR_AE, y + 1); ky1 = prof(g, 1, PR_KE, y + 1); }
  const bool yin = y >= g.P && y < g.ny - g.P;
  const bool xyin0 = v0 && yin && x >= g.P && x < g.nx - g.P;
  const bool xyin1 = v1 && yin && x + 1 >= g.P && x + 1 < g.nx - g.P;
  const bool dy_ = y >= a.dlo[1] && y < a.dhi[1];
  const int dX = a.dhi[0] - a.dlo[0], dY = a.dhi[1] - a.dlo[1];
  const int lb = (ty + 1) * B::W + 2 * tx + 4;   // own pair in a lo box
  const int hb = ty * B::W + 2 * tx;             // own pair in a hi box
  const int ob = ty * TW + 2 * tx;
  const long long nc = g.nc;
  float* const Ex = a.F;
  float* const LHx = a.L + 3 * nc;
  float* const LHy = LHx + nc;
  float* const LHz = LHy + nc;
  float* const lpB = a.psiB;
  long long q = (long long)k0 * g.plane + (long long)y * g.px + x;
  float c_hx[2] = {0.f, 0.f}, c_hy[2] = {0.f, 0.f};   // Ht(p-1) own
  // partial lam_H(p-1): own value, the -z terms and the completed x / y parts
  float c_lhx[2] = {0.f, 0.f}, c_lhy[2] = {0.f, 0.f}, c_o8[2] = {0.f, 0.f}, c_o7[2] = {0.f, 0.f};
  float c_bx[2] = {0.f, 0.f}, c_by[2] = {0.f, 0.f};
  int stg = 0;
  uint32_t par = 0;
  bool ok = true;
  for (int p = p0_; p <= p1_; ++p) {
    unsigned char* st = dsm + stg * Y::STAGE;
    if (!mbar_wait(bars + stg, par, kWaitCycles)) ok = false;
    if (!__syncthreads_and(ok)) { ring_abort<S>(bars, stg, par, p, p1_, a.err); return; }
    if (v0) {
      const float* CBb = reinterpret_cast<const float*>(st + Y::CB);
      const float* LEb = reinterpret_cast<const float*>(st + Y::LE);
      const float* Hb = reinterpret_cast<const float*>(st + Y::H);
      if (p >= k0 && p < k1) {
        const int k = p;
        const float2 cb2 = ld2(CBb, hb);
        const float2 lx2 = ld2(LEb, hb), ly2 = ld2(LEb + B::P, hb), lz2 = ld2(LEb + 2 * B::P, hb);
        const float cbv[2] = {cb2.x, cb2.y};
        const float lex[2] = {lx2.x, lx2.y}, ley[2] = {ly2.x, ly2.y}, lez[2] = {lz2.x, lz2.y};
        const bool hv = primal_plane(k) || primal_plane(k + 1);   // H box staged
        float hx[2] = {0.f, 0.f}, hy[2] = {0.f, 0.f}, hz[2] = {0.f, 0.f};
        if (hv) {
          const float2 h0 = ld2(Hb, lb), h1 = ld2(Hb + B::P, lb), h2 = ld2(Hb + 2 * B::P, lb);
          hx[0] = h0.x; hx[1] = h0.y;
          hy[0] = h1.x; hy[1] = h1.y;
          hz[0] = h2.x; hz[1] = h2.y;
        }
        // primal inverse E update on the interior, dL/dcb on the design box
        if (primal_plane(k) && (xyin0 || xyin1)) {
          const float2 hzy = ld2(Hb + 2 * B::P, lb - B::W), hxy = ld2(Hb, lb - B::W);
          const float hzx = Hb[2 * B::P + lb - 1], hyx = Hb[B::P + lb - 1];
          const float d6[2] = {hz[0] - hzy.x, hz[1] - hzy.y}, d7[2] = {hy[0] - c_hy[0], hy[1] - c_hy[1]};
          const float d8[2] = {hx[0] - c_hx[0], hx[1] - c_hx[1]}, d9[2] = {hz[0] - hzx, hz[1] - hz[0]};
          const float d10[2] = {hy[0] - hyx, hy[1] - hy[0]}, d11[2] = {hx[0] - hxy.x, hx[1] - hxy.y};
          float c0[2], c1[2], c2[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            c0[c] = d6[c] - d7[c];
            c1[c] = d8[c] - d9[c];
            c2[c] = d10[c] - d11[c];
          }
          if (a.src.kind) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const float w = (c == 0 || v1) ? src_wt(a.src, x + c, y, k) : 0.f;
              if (w != 0.f) {
                const float wj = __fmul_rn(w, a.jn);
                if (a.src.comp == 0) c0[c] = __fsub_rn(c0[c], wj);
                else if (a.src.comp == 1) c1[c] = __fsub_rn(c1[c], wj);
                else c2[c] = __fsub_rn(c2[c], wj);
              }
            }
          }
          const float* Eo = reinterpret_cast<const float*>(st + Y::E);
          const float2 e0 = ld2(Eo, ob), e1 = ld2(Eo + B::OP, ob), e2 = ld2(Eo + 2 * B::OP, ob);
          auto inc = [&](float cbc, float cc) {
            return inc_of<EX>(__fmul_rn(cbc, cc), a);
          };
          ST2(Ex, q, __fsub_rn(e0.x, inc(cbv[0], c0[0])), __fsub_rn(e0.y, inc(cbv[1], c0[1])),
              xyin0, xyin1);
          ST2(Ex + nc, q, __fsub_rn(e1.x, inc(cbv[0], c1[0])), __fsub_rn(e1.y, inc(cbv[1], c1[1])),
              xyin0, xyin1);
          ST2(Ex + 2 * nc, q, __fsub_rn(e2.x, inc(cbv[0], c2[0])),
              __fsub_rn(e2.y, inc(cbv[1], c2[1])), xyin0, xyin1);
          if (dy_ && k >= a.dlo[2] && k < a.dhi[2]) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const int xc = x + c;
              if ((c == 0 ? xyin0 : xyin1) && xc >= a.dlo[0] && xc < a.dhi[0]) {
                const float s = lex[c] * c0[c] + ley[c] * c1[c] + lez[c] * c2[c];
                const long long qd =
                    ((long long)(k - a.dlo[2]) * dY + (y - a.dlo[1])) * dX + (xc - a.dlo[0]);
                // one owner per cell: a fire-and-forget reduction in L2 adds
                // exactly what a load-add-store would, without the load latency
#ifdef FDTD_BOUNDS_CHECK
                if (qd < 0 || qd >= (long long)dX * dY * (a.dhi[2] - a.dlo[2])) {
                  atomicOr(a.err, ERR_BOUNDS);
                  continue;
                }
#endif
                atomicAdd(a.gacc + qd, (double)s);
              }
            }
          }
        }
        // adjoint of the E half-step, own and +x / +y terms
        float o6[2], o11[2], o7[2], o8[2], o9[2], o10[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float wx = cbv[c] * lex[c], wy = cbv[c] * ley[c], wz = cbv[c] * lez[c];
          o6[c] = wx; o11[c] = -wz; o7[c] = -wx; o8[c] = wy; o9[c] = -wy; o10[c] = wz;
        }
        float n6[2], n11[2];
        {
          const float2 cy2 = ld2(CBb, hb + B::W);
          const float2 ly = ld2(LEb, hb + B::W), lz = ld2(LEb + 2 * B::P, hb + B::W);
          n6[0] = cy2.x * ly.x;
          n6[1] = cy2.y * ly.y;
          n11[0] = -cy2.x * lz.x;
          n11[1] = -cy2.y * lz.y;
        }
        float n9x, n10x;   // +x terms of cell 1 (from x + 2)
        {
          const float c2 = CBb[hb + 2];
          n9x = -c2 * LEb[B::P + hb + 2];
          n10x = c2 * LEb[2 * B::P + hb + 2];
        }
        if (y + 1 >= g.ny) {
          n6[0] = 0.f; n6[1] = 0.f; n11[0] = 0.f; n11[1] = 0.f;
        }
        if (x + 2 >= g.nx) { n9x = 0.f; n10x = 0.f; }
        if (sy || sy1) {
          const float* P = reinterpret_cast<const float*>(st + Y::PY);   // TW x (TY+1) at (x0, y0)
          if (sy) {
            const float2 p0 = ld2(P, ob), p1 = ld2(P + B::YP, ob);
            const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
            float s6[2], s11[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              o6[c] = adj(o6[c], q0[c], by, ay, ky, &s6[c]);
              o11[c] = adj(o11[c], q1[c], by, ay, ky, &s11[c]);
            }
            const long long qyy = psi_ix<1>(a.pl, 2, x, y, k);
            ST2(lpB, qyy, s6[0], s6[1], true, v1);
            ST2(lpB + a.pl.ax[1].cs, qyy, s11[0], s11[1], true, v1);
          }
          if (sy1) {
            const float2 p0 = ld2(P, ob + TW), p1 = ld2(P + B::YP, ob + TW);
            const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
            float dummy;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              n6[c] = adj(n6[c], q0[c], by1, ay1, ky1, &dummy);
              n11[c] = adj(n11[c], q1[c], by1, ay1, ky1, &dummy);
            }
          }
        }
        if (sx0 || sx1 || sx2) {
          const float* P = reinterpret_cast<const float*>(st + Y::PX);   // (TW+4) x TY at (x0, y0)
          const int xb = ty * B::W + 2 * tx;
          const float2 p0 = ld2(P, xb), p1 = ld2(P + B::XP, xb);
          float s9[2] = {0.f, 0.f}, s10[2] = {0.f, 0.f};
          if (sx0) {
            o9[0] = adj(o9[0], p0.x, bx0, ax0, kx0, &s9[0]);
            o10[0] = adj(o10[0], p1.x, bx0, ax0, kx0, &s10[0]);
          }
          if (sx1) {
            o9[1] = adj(o9[1], p0.y, bx1, ax1, kx1, &s9[1]);
            o10[1] = adj(o10[1], p1.y, bx1, ax1, kx1, &s10[1]);
          }
          const long long qxx = psi_ix<0>(a.pl, 2, x, y, k);
          ST2(lpB, qxx, s9[0], s9[1], sx0, sx1);
          ST2(lpB + a.pl.ax[0].cs, qxx, s10[0], s10[1], sx0, sx1);
          if (sx2) {
            float dummy;
            n9x = adj(n9x, P[xb + 2], bx2, ax2, kx2, &dummy);
            n10x = adj(n10x, P[B::XP + xb + 2], bx2, ax2, kx2, &dummy);
          }
        }
        // cell 0's +x terms are cell 1's own terms
        const float n9[2] = {v1 ? o9[1] : 0.f, n9x}, n10[2] = {v1 ? o10[1] : 0.f, n10x};
        if (in_slab(k, g.nz, g.P)) {
          const float* P = reinterpret_cast<const float*>(st + Y::PZ);
          const float b = prof(g, 2, PR_BE, k), aa = prof(g, 2, PR_AE, k), kv = prof(g, 2, PR_KE, k);
          const float2 p0 = ld2(P, ob), p1 = ld2(P + B::OP, ob);
          const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
          float s7[2], s8[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            o7[c] = adj(o7[c], q0[c], b, aa, kv, &s7[c]);
            o8[c] = adj(o8[c], q1[c], b, aa, kv, &s8[c]);
          }
          const long long qz = psi_ix<2>(a.pl, 2, x, y, k);
          ST2(lpB, qz, s7[0], s7[1], true, v1);
          ST2(lpB + a.pl.ax[2].cs, qz, s8[0], s8[1], true, v1);
        }
        const float* LHo = reinterpret_cast<const float*>(st + Y::LH);
        const float2 lh0 = ld2(LHo, ob), lh1 = ld2(LHo + B::OP, ob), lh2 = ld2(LHo + 2 * B::OP, ob);
        ST2(LHz, q, lh2.x + ((o6[0] - n6[0]) + (o9[0] - n9[0])),
            lh2.y + ((o6[1] - n6[1]) + (o9[1] - n9[1])), true, v1);
        if (p > k0) {  // finish lam_H(p-1): its +z terms are this plane's o7, o8
          const long long qm = q - g.plane;
          ST2(LHx, qm, c_lhx[0] + ((c_o8[0] - o8[0]) + c_bx[0]), c_lhx[1] + ((c_o8[1] - o8[1]) + c_bx[1]),
              true, v1);
          ST2(LHy, qm, c_lhy[0] + ((c_o7[0] - o7[0]) + c_by[0]), c_lhy[1] + ((c_o7[1] - o7[1]) + c_by[1]),
              true, v1);
        }
        c_lhx[0] = lh0.x; c_lhx[1] = lh0.y;
        c_lhy[0] = lh1.x; c_lhy[1] = lh1.y;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          c_o8[c] = o8[c];
          c_o7[c] = o7[c];
          c_bx[c] = o11[c] - n11[c];
          c_by[c] = o10[c] - n10[c];
          c_hx[c] = hx[c];
          c_hy[c] = hy[c];
        }
        q += g.plane;
      } else if (p < k0) {
        if (primal_plane(p) || primal_plane(p + 1)) {
          const float2 h0 = ld2(Hb, lb), h1 = ld2(Hb + B::P, lb);
          c_hx[0] = h0.x; c_hx[1] = h0.y;
          c_hy[0] = h1.x; c_hy[1] = h1.y;
        }
      } else {  // p == k1 > k0: finish lam_H(k1-1) with the +z terms of plane k1
        float n7[2] = {0.f, 0.f}, n8[2] = {0.f, 0.f};
        if (p < g.nz) {
          const float2 c2 = ld2(CBb, hb), lx = ld2(LEb, hb), ly = ld2(LEb + B::P, hb);
          n7[0] = -c2.x * lx.x;
          n7[1] = -c2.y * lx.y;
          n8[0] = c2.x * ly.x;
          n8[1] = c2.y * ly.y;
          if (in_slab(p, g.nz, g.P)) {
            const float* P = reinterpret_cast<const float*>(st + Y::PZ);
            const float b1 = prof(g, 2, PR_BE, p), a1 = prof(g, 2, PR_AE, p), k1v = prof(g, 2, PR_KE, p);
            const float2 p0 = ld2(P, ob), p1 = ld2(P + B::OP, ob);
            const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
            float dummy;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              n7[c] = adj(n7[c], q0[c], b1, a1, k1v, &dummy);
              n8[c] = adj(n8[c], q1[c], b1, a1, k1v, &dummy);
            }
          }
        }
        const long long qm = q - g.plane;
        ST2(LHx, qm, c_lhx[0] + ((c_o8[0] - n8[0]) + c_bx[0]), c_lhx[1] + ((c_o8[1] - n8[1]) + c_bx[1]),
            true, v1);
        ST2(LHy, qm, c_lhy[0] + ((c_o7[0] - n7[0]) + c_by[0]), c_lhy[1] + ((c_o7[1] - n7[1]) + c_by[1]),
            true, v1);
      }
    }
    __syncthreads();
    if (tid == 0 && p + S <= p1_) issue(p + S, st, bars + stg);
    if (++stg == S) { stg = 0; par ^= 1u; }
  }
}

// ======================================== reverse H phase (+ adjoint E) ===
template <int TY, int S, int TW, bool EX, bool BM>
__global__ void __launch_bounds__(TW / 2 * TY, (min_ctas<TY, S, TW>(false)))
k_l2rev_h(const __grid_constant__ LagMaps m_, StepArgs a_) {
  const int4 bu = batch_unit<BM>(a_);
  const StepArgs& a = BM ? a_.bargs[bu.x] : a_;
  const LagMaps& m = BM ? a_.bmaps[a.bmap] : m_;
  batch_maps_acquire<BM>(m);
  typedef G<TY, TW> B;
  typedef LRH<TY, S, TW> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * (TW / 2) + tx;
  const int x0 = (BM ? bu.y : (int)blockIdx.x) * TW, y0 = (BM ? bu.z : (int)blockIdx.y) * TY;
  const int x = x0 + 2 * tx, y = y0 + ty;
  const bool v0 = x < g.nx && y < g.ny, v1 = v0 && x + 1 < g.nx;
  const int k0 = (BM ? bu.w : (int)blockIdx.z + a.zc0) * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  const bool txs = tile_in_slab(max(x0 - 1, 0), min(x0 + TW - 1, g.nx - 1), g.nx, g.P);
  const bool tys = tile_in_slab(max(y0 - 1, 0), min(y0 + TY - 1, g.ny - 1), g.ny, g.P);
  const bool tint = x0 + TW - 1 >= g.P && x0 < g.nx - g.P && y0 + TY - 1 >= g.P && y0 < g.ny - g.P;
  // plane k0-1: lam_H(k0-1) terms for the -z neighbour; planes k0..k1-1: the
  // step proper; plane p > k0 also finishes the primal Ht(p-1) with E(p).
  const int p0_ = k0 - 1, p1_ = k1;
  uint64_t* bars = ring_init<S>(dsm, Y::STAGE);
  // primal data only where the primal runs: interior tiles, planes P..nz-P-1
  // (and plane nz-P's E for the z difference of plane nz-P-1)
  auto primal_plane = [&](int p) { return tint && p >= g.P && p < g.nz - g.P; };
  int qx0, qy0;
  psi_box_starts<TW, TY>(a.pl, x0, y0, &qx0, &qy0);
  auto boxes = [&](int p, auto&& f) {
    const bool head = p < k0, body = p >= k0 && p < k1, tail = p > k0;
    const bool zs = p >= 0 && p < g.nz && in_slab(p, g.nz, g.P) && (head || body);
    const bool ebox = (body && primal_plane(p)) || (tail && primal_plane(p - 1));
    const bool hown = body && primal_plane(p);
    if (ebox) f(Y::E, &m.Fw, x0, y0, p, 0, 3 * B::P * 4);
    if (head || body) f(Y::LH, &m.Lw, x0 - 4, y0 - 1, p, 3, 3 * B::P * 4);
    if (hown) f(Y::H, &m.Fo, x0, y0, p, 3, 3 * B::OP * 4);
    if (body) f(Y::LE, &m.Lo, x0, y0, p, 0, 3 * B::OP * 4);
    if (body && txs) f(Y::PX, &m.Qxw, qx0 - 4, y0, p, 0, 2 * B::XP * 4);
    if (body && tys) f(Y::PY, &m.Qyw, x0, qy0 - 1, p, 0, 2 * B::YP * 4);
    if (zs) f(Y::PZ, &m.Qzo, x0, y0, psi_map(a.pl.ax[2], p), 0, 2 * B::OP * 4);
  };
  auto issue = [&](int p, unsigned char* st, uint64_t* bar) {
    stage_plane(boxes, p, st, bar, a.prefetch && p + 1 <= p1_ && p + 1 >= 0 && p + 1 < g.nz);
  };
  pdl_sync();
  if (tid == 0)
    for (int i = 0; i < S && p0_ + i <= p1_; ++i) issue(p0_ + i, dsm + i * Y::STAGE, bars + i);
  // x profiles at x-1 (cell 0's -x neighbour), x and x+1
  const bool sx0 = v0 && in_slab(x, g.nx, g.P), sx1 = v1 && in_slab(x + 1, g.nx, g.P);
  const bool sxm = v0 && x > 0 && in_slab(x - 1, g.nx, g.P);
  const bool sy = v0 && in_slab(y, g.ny, g.P), sym = v0 && y > 0 && in_slab(y - 1, g.ny, g.P);
  float bx0 = 0.f, ax0 = 0.f, kx0 = 1.f, bx1 = 0.f, ax1 = 0.f, kx1 = 1.f, bxm = 0.f, axm = 0.f, kxm = 1.f;
  float by = 0.f, ay = 0.f, ky = 1.f, bym = 0.f, aym = 0.f, kym = 1.f;
  if (sx0) { bx0 = prof(g, 0, PR_BH, x); ax0 = prof(g, 0, PR_AH, x); kx0 = prof(g, 0, PR_KH, x); }
  if (sx1) { bx1 = prof(g, 0, PR_BH, x + 1); ax1 = prof(g, 0, PR_AH, x + 1); kx1 = prof(g, 0, PR_KH, x + 1); }
  if (sxm) { bxm = prof(g, 0, PR_BH, x - 1); axm = prof(g, 0, PR_AH, x - 1); kxm = prof(g, 0, PR_KH, x - 1); }
  if (sy) { by = prof(g, 1, PR_BH, y); ay = prof(g, 1, PR_AH, y); ky = prof(g, 1, PR_KH, y); }
  if (sym) { bym = prof(g, 1, PR_BH, y - 1); aym = prof(g, 1, PR_AH, y - 1); kym = prof(g, 1, PR_KH, y - 1); }
  const bool yin = y >= g.P && y < g.ny - g.P;
  const bool xyin0 = v0 && yin && x >= g.P && x < g.nx - g.P;
  const bool xyin1 = v1 && yin && x + 1 >= g.P && x + 1 < g.nx - g.P;
  const int lb = (ty + 1) * B::W + 2 * tx + 4;
  const int hb = ty * B::W + 2 * tx;
  const int ob = ty * TW + 2 * tx;
  const float S_ = g.S;
  const long long nc = g.nc;
  float* const Hx = a.F + 3 * nc;
  float* const LEx = a.L;
  float* const lpB = a.psiB;
  long long q = (long long)k0 * g.plane + (long long)y * g.px + x;
  float c_m1[2] = {0.f, 0.f}, c_m2[2] = {0.f, 0.f};   // -z neighbour terms from plane p-1
  float c_d0[2] = {0.f, 0.f}, c_d3[2] = {0.f, 0.f}, c_d4[2] = {0.f, 0.f}, c_d5[2] = {0.f, 0.f};
  float c_ex[2] = {0.f, 0.f}, c_ey[2] = {0.f, 0.f};
  float c_hx[2] = {0.f, 0.f}, c_hy[2] = {0.f, 0.f}, c_hz[2] = {0.f, 0.f};
  bool c_pr0 = false, c_pr1 = false;   // primal Ht(p-1) pending per cell
  int stg = 0;
  uint32_t par = 0;
  bool ok = true;
  for (int p = p0_; p <= p1_; ++p) {
    unsigned char* st = dsm + stg * Y::STAGE;
    if (!mbar_wait(bars + stg, par, kWaitCycles)) ok = false;
    if (!__syncthreads_and(ok)) { ring_abort<S>(bars, stg, par, p, p1_, a.err); return; }
    if (v0) {
      const float* Eb = reinterpret_cast<const float*>(st + Y::E);
      if (p > k0 && (c_pr0 || c_pr1)) {  // finish the primal Ht(p-1) with dEy/dz, dEx/dz
        const float2 ex = ld2(Eb, hb), ey = ld2(Eb + B::P, hb);
        const float d1[2] = {ey.x - c_ey[0], ey.y - c_ey[1]};
        const float d2[2] = {ex.x - c_ex[0], ex.y - c_ex[1]};
        const long long qm = q - g.plane;
        auto inc = [&](float cc) { return inc_of<EX>(__fmul_rn(S_, cc), a); };
        ST2(Hx, qm, __fadd_rn(c_hx[0], inc(c_d0[0] - d1[0])),
            __fadd_rn(c_hx[1], inc(c_d0[1] - d1[1])), c_pr0, c_pr1);
        ST2(Hx + nc, qm, __fadd_rn(c_hy[0], inc(d2[0] - c_d3[0])),
            __fadd_rn(c_hy[1], inc(d2[1] - c_d3[1])), c_pr0, c_pr1);
        ST2(Hx + 2 * nc, qm, __fadd_rn(c_hz[0], inc(c_d4[0] - c_d5[0])),
            __fadd_rn(c_hz[1], inc(c_d4[1] - c_d5[1])), c_pr0, c_pr1);
      }
      const float* LHb = reinterpret_cast<const float*>(st + Y::LH);
      if (p >= k0 && p < k1) {
        const int k = p;
        const bool pp = primal_plane(k);
        c_pr0 = pp && xyin0;
        c_pr1 = pp && xyin1;
        if (c_pr0 || c_pr1) {  // primal Ht(k): x and y derivatives now, z derivatives next plane
          const float2 ex = ld2(Eb, hb), ey = ld2(Eb + B::P, hb), ez = ld2(Eb + 2 * B::P, hb);
          const float2 ezy = ld2(Eb + 2 * B::P, hb + B::W), exy = ld2(Eb, hb + B::W);
          const float ezx = Eb[2 * B::P + hb + 2], eyx = Eb[B::P + hb + 2];
          const float* Ho = reinterpret_cast<const float*>(st + Y::H);
          const float2 h0 = ld2(Ho, ob), h1 = ld2(Ho + B::OP, ob), h2 = ld2(Ho + 2 * B::OP, ob);
          c_d0[0] = ezy.x - ez.x; c_d0[1] = ezy.y - ez.y;
          c_d3[0] = ez.y - ez.x;  c_d3[1] = ezx - ez.y;
          c_d4[0] = ey.y - ey.x;  c_d4[1] = eyx - ey.y;
          c_d5[0] = exy.x - ex.x; c_d5[1] = exy.y - ex.y;
          c_ex[0] = ex.x; c_ex[1] = ex.y;
          c_ey[0] = ey.x; c_ey[1] = ey.y;
          c_hx[0] = h0.x; c_hx[1] = h0.y;
          c_hy[0] = h1.x; c_hy[1] = h1.y;
          c_hz[0] = h2.x; c_hz[1] = h2.y;
        }
        // adjoint of the H half-step: lam_E += D^T lam_delta, v = -S s lam_H
        const float2 lx2 = ld2(LHb, lb), ly2 = ld2(LHb + B::P, lb), lz2 = ld2(LHb + 2 * B::P, lb);
        const float lhx[2] = {lx2.x, lx2.y}, lhy[2] = {ly2.x, ly2.y}, lhz[2] = {lz2.x, lz2.y};
        float o0[2], o1[2], o2[2], o3[2], o4[2], o5[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          o0[c] = -S_ * lhx[c];
          o5[c] = S_ * lhz[c];
          o1[c] = S_ * lhx[c];
          o2[c] = -S_ * lhy[c];
          o3[c] = S_ * lhy[c];
          o4[c] = -S_ * lhz[c];
        }
        float m0[2], m5[2];
        {
          const float2 lxy = ld2(LHb, lb - B::W), lzy = ld2(LHb + 2 * B::P, lb - B::W);   // -y
          m0[0] = -S_ * lxy.x; m0[1] = -S_ * lxy.y;
          m5[0] = S_ * lzy.x;  m5[1] = S_ * lzy.y;
        }
        float m3x = S_ * LHb[B::P + lb - 1], m4x = -S_ * LHb[2 * B::P + lb - 1];   // -x of cell 0
        if (y == 0) { m0[0] = 0.f; m0[1] = 0.f; m5[0] = 0.f; m5[1] = 0.f; }
        if (x == 0) { m3x = 0.f; m4x = 0.f; }
        if (sy || sym) {
          const float* P = reinterpret_cast<const float*>(st + Y::PY);   // TW x (TY+1) at (x0, y0-1)
          const int yb = (ty + 1) * TW + 2 * tx;
          if (sy) {
            const float2 p0 = ld2(P, yb), p1 = ld2(P + B::YP, yb);
            const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
            float s4[2], s5[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              o0[c] = adj(o0[c], q0[c], by, ay, ky, &s4[c]);
              o5[c] = adj(o5[c], q1[c], by, ay, ky, &s5[c]);
            }
            const long long qyy = psi_ix<1>(a.pl, 0, x, y, k);
            ST2(lpB, qyy, s4[0], s4[1], true, v1);
            ST2(lpB + a.pl.ax[1].cs, qyy, s5[0], s5[1], true, v1);
          }
          if (sym) {
            const float2 p0 = ld2(P, yb - TW), p1 = ld2(P + B::YP, yb - TW);
            const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
            float dummy;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              m0[c] = adj(m0[c], q0[c], bym, aym, kym, &dummy);
              m5[c] = adj(m5[c], q1[c], bym, aym, kym, &dummy);
            }
          }
        }
        if (sx0 || sx1 || sxm) {
          const float* P = reinterpret_cast<const float*>(st + Y::PX);   // (TW+4) x TY at (x0-4, y0)
          const int xb = ty * B::W + 2 * tx + 4;
          const float2 p0 = ld2(P, xb), p1 = ld2(P + B::XP, xb);
          float s0[2] = {0.f, 0.f}, s1[2] = {0.f, 0.f};
          if (sx0) {
            o3[0] = adj(o3[0], p0.x, bx0, ax0, kx0, &s0[0]);
            o4[0] = adj(o4[0], p1.x, bx0, ax0, kx0, &s1[0]);
          }
          if (sx1) {
            o3[1] = adj(o3[1], p0.y, bx1, ax1, kx1, &s0[1]);
            o4[1] = adj(o4[1], p1.y, bx1, ax1, kx1, &s1[1]);
          }
          const long long qxx = psi_ix<0>(a.pl, 0, x, y, k);
          ST2(lpB, qxx, s0[0], s0[1], sx0, sx1);
          ST2(lpB + a.pl.ax[0].cs, qxx, s1[0], s1[1], sx0, sx1);
          if (sxm) {
            float dummy;
            m3x = adj(m3x, P[xb - 1], bxm, axm, kxm, &dummy);
            m4x = adj(m4x, P[B::XP + xb - 1], bxm, axm, kxm, &dummy);
          }
        }
        // cell 1's -x terms are cell 0's own terms
        const float m3[2] = {m3x, o3[0]}, m4[2] = {m4x, o4[0]};
        if (in_slab(k, g.nz, g.P)) {
          const float* P = reinterpret_cast<const float*>(st + Y::PZ);
          const float b = prof(g, 2, PR_BH, k), aa = prof(g, 2, PR_AH, k), kv = prof(g, 2, PR_KH, k);
          const float2 p0 = ld2(P, ob), p1 = ld2(P + B::OP, ob);
          const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
          float s8[2], s9[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            o1[c] = adj(o1[c], q0[c], b, aa, kv, &s8[c]);
            o2[c] = adj(o2[c], q1[c], b, aa, kv, &s9[c]);
          }
          const long long qz = psi_ix<2>(a.pl, 0, x, y, k);
          ST2(lpB, qz, s8[0], s8[1], true, v1);
          ST2(lpB + a.pl.ax[2].cs, qz, s9[0], s9[1], true, v1);
        }
        const float* LEo = reinterpret_cast<const float*>(st + Y::LE);
        const float2 le0 = ld2(LEo, ob), le1 = ld2(LEo + B::OP, ob), le2 = ld2(LEo + 2 * B::OP, ob);
        ST2(LEx, q, le0.x + ((c_m2[0] - o2[0]) + (m5[0] - o5[0])),
            le0.y + ((c_m2[1] - o2[1]) + (m5[1] - o5[1])), true, v1);
        ST2(LEx + nc, q, le1.x + ((c_m1[0] - o1[0]) + (m4[0] - o4[0])),
            le1.y + ((c_m1[1] - o1[1]) + (m4[1] - o4[1])), true, v1);
        ST2(LEx + 2 * nc, q, le2.x + ((m0[0] - o0[0]) + (m3[0] - o3[0])),
            le2.y + ((m0[1] - o0[1]) + (m3[1] - o3[1])), true, v1);
        // the -z terms plane p+1 needs are this plane's own z-terms
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          c_m1[c] = o1[c];
          c_m2[c] = o2[c];
        }
        q += g.plane;
      } else if (p < k0) {  // -z terms for plane k0 from plane k0-1
        float m1n[2] = {0.f, 0.f}, m2n[2] = {0.f, 0.f};
        if (p >= 0) {
          const float2 lx2 = ld2(LHb, lb), ly2 = ld2(LHb + B::P, lb);
          m1n[0] = S_ * lx2.x; m1n[1] = S_ * lx2.y;
          m2n[0] = -S_ * ly2.x; m2n[1] = -S_ * ly2.y;
          if (in_slab(p, g.nz, g.P)) {
            const float* P = reinterpret_cast<const float*>(st + Y::PZ);
            const float b1 = prof(g, 2, PR_BH, p), a1 = prof(g, 2, PR_AH, p), k1v = prof(g, 2, PR_KH, p);
            const float2 p0 = ld2(P, ob), p1 = ld2(P + B::OP, ob);
            const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
            float dummy;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              m1n[c] = adj(m1n[c], q0[c], b1, a1, k1v, &dummy);
              m2n[c] = adj(m2n[c], q1[c], b1, a1, k1v, &dummy);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          c_m1[c] = m1n[c];
          c_m2[c] = m2n[c];
        }
      }
    }
    __syncthreads();
    if (tid == 0 && p + S <= p1_) issue(p + S, st, bars + stg);
    if (++stg == S) { stg = 0; par ^= 1u; }
  }
}

// ------------------------------------------------------------ launchers ---
template <class KT>
static cudaError_t set_smem_l2(KT kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Launch with the programmatic-stream-serialization attribute when a.pdl is
// set (the kernel then overlaps its launch and prologue with the tail of the
// previous kernel and waits in pdl_sync()).
template <class KT>
static cudaError_t launch_ex(KT kernel, dim3 grid, dim3 block, int smem, cudaStream_t s,
                             const LagMaps& m, const StepArgs& a) {
  cudaError_t e = set_smem_l2(kernel, smem);
  if (e) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = a.pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, m, a);
}

template <int TY, int S, int TW = 32, bool EX = false>
static cudaError_t launch_lag2_t(int which, const LagMaps& m, const StepArgs& a, cudaStream_t s) {
  static_assert((TW / 2 * TY) % 32 == 0, "a CTA is a whole number of warps");
  if constexpr (TY == 8 && TW == 32 && S == 2 && !EX) {
    if (a.bunits) {   // batched designs: one CTA per listed unit
      if (a.bcount <= 0) return cudaSuccess;
      const dim3 bg((unsigned)a.bcount, 1, 1), blk(TW / 2, TY);
      switch (which) {
        case 0: return launch_ex(k_l2fwd_h<TY, S, TW, EX, false, true>, bg, blk, LFH<TY, S, TW>::smem(), s, m, a);
        case 1: return launch_ex(k_l2fwd_e<TY, S, TW, EX, false, true>, bg, blk, LFE<TY, S, TW>::smem(), s, m, a);
        case 2: return launch_ex(k_l2rev_e<TY, S, TW, EX, true>, bg, blk, LRE<TY, S, TW>::smem(), s, m, a);
        case 3: return launch_ex(k_l2rev_h<TY, S, TW, EX, true>, bg, blk, LRH<TY, S, TW>::smem(), s, m, a);
      }
      return cudaErrorInvalidValue;
    }
  }
  if (a.bunits) return cudaErrorInvalidValue;   // batched designs: 32 x 8 tiles, two stages
  const int nch = (a.g.nz + a.zchunk - 1) / a.zchunk;
  const int zc1 = a.zc1 > 0 ? min(a.zc1, nch) : nch;
  if (a.zc0 < 0 || a.zc0 >= zc1) return cudaErrorInvalidValue;
  dim3 grid((a.g.nx + TW - 1) / TW, (a.g.ny + TY - 1) / TY, zc1 - a.zc0);
  if (a.umode) {   // the forward half-steps over the CPML units of a fused forward step
    if (which > 1 || TY != 8 || TW != 32 || a.U.nzc != nch) return cudaErrorInvalidValue;
    const RevUnits& U = a.U;
    grid = a.umode == 1 ? dim3(U.ix1 - U.ix0, U.iy1 - U.iy0, U.nzc - (U.iz1 - U.iz0))
                        : dim3((unsigned)(ring_tiles(U) * U.nzc), 1, 1);
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
  }
  dim3 block(TW / 2, TY);
  if constexpr (TY == 8 && TW == 32) {
    if (a.umode) {
      if (!a.Fn) return cudaErrorInvalidValue;
      if (which == 0)
        return launch_ex(k_l2fwd_h<TY, S, TW, EX, true, false>, grid, block, LFH<TY, S, TW>::smem(), s, m, a);
      return launch_ex(k_l2fwd_e<TY, S, TW, EX, true, false>, grid, block, LFE<TY, S, TW>::smem(), s, m, a);
    }
  }
  switch (which) {
    case 0: return launch_ex(k_l2fwd_h<TY, S, TW, EX, false, false>, grid, block, LFH<TY, S, TW>::smem(), s, m, a);
    case 1: return launch_ex(k_l2fwd_e<TY, S, TW, EX, false, false>, grid, block, LFE<TY, S, TW>::smem(), s, m, a);
    case 2: return launch_ex(k_l2rev_e<TY, S, TW, EX, false>, grid, block, LRE<TY, S, TW>::smem(), s, m, a);
    case 3: return launch_ex(k_l2rev_h<TY, S, TW, EX, false>, grid, block, LRH<TY, S, TW>::smem(), s, m, a);
  }
  return cudaErrorInvalidValue;
}

// which: 0 forward H, 1 forward E, 2 reverse E phase, 3 reverse H phase.
// Exact reversal (a.xq != 0) runs 32 x 8 tiles with two stages.  A warp covers two tile rows, so tile heights start at 2 (the caller runs
// a requested height of 1 as 2).  Stage counts 2 and 4 are built for tile
// heights 2, 4 and 8; height 16 runs with 3.
cudaError_t launch_lag2(int which, const LagMaps& m, const StepArgs& a, cudaStream_t s) {
  const int S = a.stages;
  if (a.xq) {   // exact reversal: built for the default shape only
    if (a.tile_y != 8 || S != 2 || a.tile_x != 32) return cudaErrorInvalidValue;
    return launch_lag2_t<8, 2, 32, true>(which, m, a, s);
  }
  if (a.tile_x == 40) {   // 40-wide tiles: tile height 8 only (whole warps), 2 or 3 stages
    if (a.tile_y != 8) return cudaErrorInvalidValue;
    return S == 3 ? launch_lag2_t<8, 3, 40>(which, m, a, s) : launch_lag2_t<8, 2, 40>(which, m, a, s);
  }
  switch (a.tile_y) {
    case 2: return S == 2 ? launch_lag2_t<2, 2>(which, m, a, s)
                 : S == 4 ? launch_lag2_t<2, 4>(which, m, a, s) : launch_lag2_t<2, 3>(which, m, a, s);
    case 4: return S == 2 ? launch_lag2_t<4, 2>(which, m, a, s)
                 : S == 4 ? launch_lag2_t<4, 4>(which, m, a, s) : launch_lag2_t<4, 3>(which, m, a, s);
    case 8: return S == 2 ? launch_lag2_t<8, 2>(which, m, a, s)
                 : S == 4 ? launch_lag2_t<8, 4>(which, m, a, s) : launch_lag2_t<8, 3>(which, m, a, s);
    case 16: return launch_lag2_t<16, 3>(which, m, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fdtd
