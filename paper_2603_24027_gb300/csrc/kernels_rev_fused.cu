// kernels_rev_fused.cu -- one reverse time step in two fused launches.
//
// A reverse step n (Sec. 2: the time-reversed interior with the adjoint run
// alongside) starts from E^{n+1}, Ht^{n+1/2} with the interface layers
// restored and from the adjoint fields after the objective seed.  The split
// kernels (kernels_lag2.cu) run it as two phases that each read and write
// both the primal and the adjoint fields (148 B per interior cell); here it
// is two launches that each run BOTH half-steps of one family, reading every
// field once and writing it once:
//
//   primal  (k_rev_primal, interior cells only):
//       E^n        = E^{n+1} - cb (curl Ht^{n+1/2} - J)
//       Ht^{n-1/2} = Ht^{n+1/2} + S curl E^n
//     and the design-box accumulation dL/dcb += lam_E^{n+1} . (curl Ht - J);
//   adjoint (k_rev_adjoint, every cell, CPML auxiliaries included):
//       lam_H' = lam_H + C_H^T (cb lam_E)      (transpose of the E half-step)
//       lam_E' = lam_E - C_E^T (S lam_H')      (transpose of the H half-step)
//
// 52 B per interior cell each (cb is read by both), 52 B per CPML cell for
// the adjoint.  Both kernels read the current buffer of each field and write
// the other one of a ping-pong pair, so no CTA can read a value another CTA
// of the same launch has already replaced; the two launches are independent
// of each other within a step.
//
// Each CTA owns a 32 x TY column tile and a z chunk, staged plane by plane
// with TMA box loads into a ring of shared-memory stages, as in the split
// kernels.  The second half-step of a plane needs the first half-step's
// results on the neighbouring cells: E^n at +x / +y (primal), lam_H' at -x /
// -y (adjoint).  Across z they come one iteration later (the second
// half-step lags one plane); across x and y the CTA computes them itself on
// a one-cell halo of its tile, from the same staged inputs, with the same
// sequence of rounded operations as the cell's owner.  Four warps own the
// tile's pairs of cells; a fifth computes the halo (a row of 16 pairs and a
// column of TY cells).  The primal half-steps repeat the forward's rounded
// operations exactly, so the primal fields are bit-identical to the split
// kernels'; the adjoint sums are left to the compiler's contraction, as in
// the split kernels.
#include <cudaTypedefs.h>

#include "lag_common.cuh"

namespace fdtd {

using namespace lag2;

namespace revf {

// Shared memory of the primal kernel (byte offsets): S stages of an Ht box
// (TW+8) x (TY+2) at (x0-4, y0-1) and E and cb boxes (TW+4) x (TY+1) at
// (x0, y0); the stages' mbarriers right after them (where ring_init puts
// them); then E^n of the plane on the tile and its +x / +y halo,
// [3][TY+1][TW+4] at (x0, y0).
template <int TY, int S, int TW>
struct PL {
  static constexpr int HW = TW + 8, HR = TY + 2, HP = HW * HR;
  static constexpr int EW = TW + 4, ER = TY + 1, EP = EW * ER;
  static constexpr int H = 0;
  static constexpr int E = r128(3 * HP * 4);
  static constexpr int CB = E + r128(3 * EP * 4);
  static constexpr int STAGE = CB + r128(EP * 4);
  static constexpr int BARS = S * STAGE;
  static constexpr int SE = r128(BARS + 8 * S);
  static int smem() { return SE + 3 * EP * 4; }
};

// Stage layout of the adjoint kernel: cb and lam_E boxes (TW+8) x (TY+2) at
// (x0-4, y0-1), lam_H box (TW+4) x (TY+1) at (x0-4, y0-1); with CPML terms
// (by MODE below), the adjoint auxiliaries of the E half-step at plane p (x: (TW+8) x (TY+1)
// at (x0-4, y0-1); y: (TW+4) x (TY+2) at (x0-4, y0-1); z: (TW+4) x (TY+1) at
// (x0-4, y0-1)) and of the H half-step at plane p-1 (x: (TW+4) x TY at
// (x0-4, y0); y: TW x (TY+1) at (x0, y0-1); z: TW x TY at (x0, y0)).  The
// stages' mbarriers follow the S stages; then lam_H' of plane p-1 on the
// tile and its -x / -y halo, [3][TY+1][TW+4] at (x0-4, y0-1).
// MODE 0: no CPML term in the unit; 1: z CPML terms only (tiles inside the
// x / y interior, chunks touching a z slab); 2: every axis (the x / y ring).
template <int TY, int S, int TW, int MODE>
struct AL {
  static constexpr bool PXY = MODE == 2, PZ = MODE >= 1;
  static constexpr int WW = TW + 8, WR = TY + 2, WP = WW * WR;
  static constexpr int HW = TW + 4, HR = TY + 1, HP = HW * HR;
  static constexpr int EXP = (TW + 8) * (TY + 1), EYP = (TW + 4) * (TY + 2), EZP = HP;
  static constexpr int HXP = (TW + 4) * TY, HYP = TW * (TY + 1), HZP = TW * TY;
  static constexpr int CB = 0;
  static constexpr int LE = CB + r128(WP * 4);
  static constexpr int LH = LE + r128(3 * WP * 4);
  static constexpr int PEX = LH + r128(3 * HP * 4);
  static constexpr int PEY = PEX + (PXY ? r128(2 * EXP * 4) : 0);
  static constexpr int PEZ = PEY + (PXY ? r128(2 * EYP * 4) : 0);
  static constexpr int PHX = PEZ + (PZ ? r128(2 * EZP * 4) : 0);
  static constexpr int PHY = PHX + (PXY ? r128(2 * HXP * 4) : 0);
  static constexpr int PHZ = PHY + (PXY ? r128(2 * HYP * 4) : 0);
  static constexpr int STAGE = PHZ + (PZ ? r128(2 * HZP * 4) : 0);
  static constexpr int BARS = S * STAGE;
  static constexpr int SL = r128(BARS + 8 * S);
  // ring units: the x / y CPML profiles of the tile's cells and halo
  static constexpr int SP = SL + r128(3 * HP * 4), SPXN = TW + 8, SPYN = TY + 4;
  static int smem() { return PXY ? SP + 6 * (SPXN + SPYN) * 4 : SL + 3 * HP * 4; }
};

// ring_init puts the barriers at S * STAGE: the exchange arrays come after them
static_assert(PL<8, 3, 32>::BARS == 3 * PL<8, 3, 32>::STAGE &&
              PL<8, 3, 32>::SE >= PL<8, 3, 32>::BARS + 8 * 3, "SE after the barriers");
static_assert(AL<8, 3, 32, 0>::SL >= AL<8, 3, 32, 0>::BARS + 8 * 3, "SL after the barriers");
static_assert(AL<8, 3, 32, 1>::SL >= AL<8, 3, 32, 1>::BARS + 8 * 3, "SL after the barriers");
static_assert(AL<8, 2, 32, 2>::SL >= AL<8, 2, 32, 2>::BARS + 8 * 2, "SL after the barriers");

// Resident CTAs per SM the register allocation must allow (what the shared
// memory of the default shapes allows).
template <int S, int MODE>
constexpr int adj_ctas() { return MODE == 2 ? 4 : (MODE == 1 ? 4 : 5); }

// Tile and chunk of a unit.  Primal and CPML-free adjoint launches: a 3D
// grid offset by (t0x, t0y, zc0).  z-only units (MODE 1): a 3D grid over the
// tiles [ix0, ix1) x [iy0, iy1) and the chunks outside [iz0, iz1)
// (zonly_chunk).  Ring units (MODE 2): a 1D grid over every chunk times the
// ring tiles (ring_unit).

}  // namespace revf

using namespace revf;

// ============================================================== primal ===
template <int TY, int S, int TW, bool EX>
__global__ void __launch_bounds__(TW / 2 * (TY + 2), 6)
k_rev_primal(const __grid_constant__ RevMaps m, StepArgs a) {
  typedef PL<TY, S, TW> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * (TW / 2) + tx;
  const int x0 = (blockIdx.x + a.t0x) * TW, y0 = (blockIdx.y + a.t0y) * TY;
  const int k0 = (blockIdx.z + a.zc0) * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  // task of this thread: the tile's pair (main), a pair of the +y halo row,
  // or a cell of the +x halo column (as the first cell of a pair)
  const bool mainT = ty < TY;
  const bool rowT = ty == TY;
  const bool colT = ty == TY + 1 && tx < TY;
  const bool task = mainT || rowT || colT;
  const int x = colT ? x0 + TW : x0 + 2 * tx;
  const int y = mainT ? y0 + ty : (rowT ? y0 + TY : y0 + tx);
  const bool rowok = y < g.ny;
  const bool in0 = task && rowok && x < g.nx && x >= g.P && x < g.nx - g.P && y >= g.P &&
                   y < g.ny - g.P;
  const bool in1 = task && !colT && rowok && x + 1 < g.nx && x + 1 >= g.P &&
                   x + 1 < g.nx - g.P && y >= g.P && y < g.ny - g.P;
  auto primal_plane = [&](int p) { return p >= g.P && p < g.nz - g.P; };
  const int p0_ = k0 - 1, p1_ = k1;
  uint64_t* bars = ring_init<S>(dsm, Y::STAGE);   // at Y::BARS
  // plane p >= k0 provides E^n(p): computed where p is interior, else the
  // restored layer (for Ht^{n-1/2}(p-1)); Ht(p) also carries its x, y
  // components to plane p + 1
  auto boxes = [&](int p, auto&& f) {
    const bool head = p < k0, tail = p == k1;
    const bool pp = primal_plane(p), pm = primal_plane(p - 1), pn = primal_plane(p + 1);
    const bool hbox = head ? pn : (pp || (!tail && pn));
    const bool ebox = !head && (pp || pm);
    const bool cbox = !head && pp;
    if (hbox) f(Y::H, &m.F40, x0 - 4, y0 - 1, p, 3, 3 * Y::HP * 4);
    if (ebox) f(Y::E, &m.F36, x0, y0, p, 0, 3 * Y::EP * 4);
    if (cbox) f(Y::CB, &m.cb36, x0, y0, p, 0, Y::EP * 4);
  };
  auto issue = [&](int p, unsigned char* st, uint64_t* bar) {
    stage_plane(boxes, p, st, bar, false);
  };
  if (tid == 0)
    for (int i = 0; i < S && p0_ + i <= p1_; ++i) issue(p0_ + i, dsm + i * Y::STAGE, bars + i);
  const int hb = (y - y0 + 1) * Y::HW + (x - x0 + 4);   // the pair in the Ht box
  const int eb = (y - y0) * Y::EW + (x - x0);           // the pair in the E / cb boxes and SE
  float* SE = reinterpret_cast<float*>(dsm + Y::SE);
  const long long nc = g.nc;
  float* const Fn = a.Fn;
  const bool dy_ = y >= a.dlo[1] && y < a.dhi[1];
  const int dX = a.dhi[0] - a.dlo[0], dY = a.dhi[1] - a.dlo[1];
  long long q = (long long)k0 * g.plane + (long long)y * g.px + x;   // plane k0 of the pair
  float c_hx[2] = {0.f, 0.f}, c_hy[2] = {0.f, 0.f};   // Ht^{n+1/2}(p-1) x, y at the pair
  // primal Ht^{n-1/2}(p-1) pending: the x / y differences of E^n(p-1), E^n(p-1) x, y
  // and Ht^{n+1/2}(p-1)
  float c_d0[2] = {0.f, 0.f}, c_d3[2] = {0.f, 0.f}, c_d4[2] = {0.f, 0.f}, c_d5[2] = {0.f, 0.f};
  float c_ex[2] = {0.f, 0.f}, c_ey[2] = {0.f, 0.f};
  float c_h0[2] = {0.f, 0.f}, c_h1[2] = {0.f, 0.f}, c_h2[2] = {0.f, 0.f};
  bool c_pr0 = false, c_pr1 = false;
  int stg = 0;
  uint32_t par = 0;
  bool ok = true;
  for (int p = p0_; p <= p1_; ++p) {
    unsigned char* st = dsm + stg * Y::STAGE;
    if (!mbar_wait(bars + stg, par, kWaitCycles)) ok = false;
    if (!__syncthreads_and(ok)) { ring_abort<S>(bars, stg, par, p, p1_, a.err); return; }
    const float* Hb = reinterpret_cast<const float*>(st + Y::H);
    const float* Eb = reinterpret_cast<const float*>(st + Y::E);
    const float* CBb = reinterpret_cast<const float*>(st + Y::CB);
    const bool head = p < k0, tail = p == k1;
    // ---- first half-step: E^n(p) on the task's cells ----
    float en0[2] = {0.f, 0.f}, en1[2] = {0.f, 0.f}, en2[2] = {0.f, 0.f};
    const bool need_e = !head && (primal_plane(p) || primal_plane(p - 1)) && (mainT || !tail);
    if (task && need_e) {
      const float2 e0 = ld2(Eb, eb), e1 = ld2(Eb + Y::EP, eb), e2 = ld2(Eb + 2 * Y::EP, eb);
      en0[0] = e0.x; en0[1] = e0.y;
      en1[0] = e1.x; en1[1] = e1.y;
      en2[0] = e2.x; en2[1] = e2.y;
      const bool pp = primal_plane(p);
      const bool i0 = in0 && pp, i1 = in1 && pp;
      if (i0 || i1) {
        const float2 hx = ld2(Hb, hb), hy = ld2(Hb + Y::HP, hb), hz = ld2(Hb + 2 * Y::HP, hb);
        const float2 hzy = ld2(Hb + 2 * Y::HP, hb - Y::HW), hxy = ld2(Hb, hb - Y::HW);
        const float hzx = Hb[2 * Y::HP + hb - 1], hyx = Hb[Y::HP + hb - 1];
        const float d6[2] = {hz.x - hzy.x, hz.y - hzy.y}, d7[2] = {hy.x - c_hy[0], hy.y - c_hy[1]};
        const float d8[2] = {hx.x - c_hx[0], hx.y - c_hx[1]}, d9[2] = {hz.x - hzx, hz.y - hz.x};
        const float d10[2] = {hy.x - hyx, hy.y - hy.x}, d11[2] = {hx.x - hxy.x, hx.y - hxy.y};
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
            const float w = (c == 0 ? i0 : i1) ? src_wt(a.src, x + c, y, p) : 0.f;
            if (w != 0.f) {
              const float wj = __fmul_rn(w, a.jn);
              if (a.src.comp == 0) c0[c] = __fsub_rn(c0[c], wj);
              else if (a.src.comp == 1) c1[c] = __fsub_rn(c1[c], wj);
              else c2[c] = __fsub_rn(c2[c], wj);
            }
          }
        }
        const float2 cb2 = ld2(CBb, eb);
        const float cbv[2] = {cb2.x, cb2.y};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (c == 0 ? i0 : i1) {
            en0[c] = __fsub_rn(en0[c], inc_of<EX>(__fmul_rn(cbv[c], c0[c]), a));
            en1[c] = __fsub_rn(en1[c], inc_of<EX>(__fmul_rn(cbv[c], c1[c]), a));
            en2[c] = __fsub_rn(en2[c], inc_of<EX>(__fmul_rn(cbv[c], c2[c]), a));
          }
        }
        if (mainT && !tail) {
          ST2(Fn, q, en0[0], en0[1], i0, i1);
          ST2(Fn + nc, q, en1[0], en1[1], i0, i1);
          ST2(Fn + 2 * nc, q, en2[0], en2[1], i0, i1);
          // dL/dcb on the design box: lam_E^{n+1} . (curl Ht - J)
          if (dy_ && p >= a.dlo[2] && p < a.dhi[2]) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const int xc = x + c;
              if ((c == 0 ? i0 : i1) && xc >= a.dlo[0] && xc < a.dhi[0]) {
                const long long qc = q + c;
                const float s = a.L[qc] * c0[c] + a.L[nc + qc] * c1[c] + a.L[2 * nc + qc] * c2[c];
                const long long qd =
                    ((long long)(p - a.dlo[2]) * dY + (y - a.dlo[1])) * dX + (xc - a.dlo[0]);
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
      }
      if (!tail && primal_plane(p)) {
        *reinterpret_cast<float2*>(SE + eb) = make_float2(en0[0], en0[1]);
        *reinterpret_cast<float2*>(SE + Y::EP + eb) = make_float2(en1[0], en1[1]);
        *reinterpret_cast<float2*>(SE + 2 * Y::EP + eb) = make_float2(en2[0], en2[1]);
      }
    }
    // Ht^{n+1/2}(p) x, y at the task's cells for the next plane's z differences
    if (task && !tail && (head ? primal_plane(p + 1) : (primal_plane(p) || primal_plane(p + 1)))) {
      const float2 hx = ld2(Hb, hb), hy = ld2(Hb + Y::HP, hb);
      c_hx[0] = hx.x; c_hx[1] = hx.y;
      c_hy[0] = hy.x; c_hy[1] = hy.y;
    }
    __syncthreads();   // E^n(p) of the tile and its halo is in SE
    // ---- second half-step, one plane behind: Ht^{n-1/2}(p-1) ----
    if (mainT && !head) {
      if (p > k0 && (c_pr0 || c_pr1)) {
        const float d1[2] = {en1[0] - c_ey[0], en1[1] - c_ey[1]};
        const float d2[2] = {en0[0] - c_ex[0], en0[1] - c_ex[1]};
        const long long qm = q - g.plane;
        auto inc = [&](float cc) { return inc_of<EX>(__fmul_rn(g.S, cc), a); };
        ST2(Fn + 3 * nc, qm, __fadd_rn(c_h0[0], inc(c_d0[0] - d1[0])),
            __fadd_rn(c_h0[1], inc(c_d0[1] - d1[1])), c_pr0, c_pr1);
        ST2(Fn + 4 * nc, qm, __fadd_rn(c_h1[0], inc(d2[0] - c_d3[0])),
            __fadd_rn(c_h1[1], inc(d2[1] - c_d3[1])), c_pr0, c_pr1);
        ST2(Fn + 5 * nc, qm, __fadd_rn(c_h2[0], inc(c_d4[0] - c_d5[0])),
            __fadd_rn(c_h2[1], inc(c_d4[1] - c_d5[1])), c_pr0, c_pr1);
      }
      if (!tail) {
        const bool pp = primal_plane(p);
        c_pr0 = pp && in0;
        c_pr1 = pp && in1;
        if (c_pr0 || c_pr1) {   // x and y differences of E^n(p) now, z differences next plane
          const float2 ezy = ld2(SE + 2 * Y::EP, eb + Y::EW), exy = ld2(SE, eb + Y::EW);
          const float ezx = SE[2 * Y::EP + eb + 2], eyx = SE[Y::EP + eb + 2];
          c_d0[0] = ezy.x - en2[0]; c_d0[1] = ezy.y - en2[1];
          c_d3[0] = en2[1] - en2[0]; c_d3[1] = ezx - en2[1];
          c_d4[0] = en1[1] - en1[0]; c_d4[1] = eyx - en1[1];
          c_d5[0] = exy.x - en0[0]; c_d5[1] = exy.y - en0[1];
          c_ex[0] = en0[0]; c_ex[1] = en0[1];
          c_ey[0] = en1[0]; c_ey[1] = en1[1];
          const float2 h0 = ld2(Hb, hb), h1 = ld2(Hb + Y::HP, hb), h2 = ld2(Hb + 2 * Y::HP, hb);
          c_h0[0] = h0.x; c_h0[1] = h0.y;
          c_h1[0] = h1.x; c_h1[1] = h1.y;
          c_h2[0] = h2.x; c_h2[1] = h2.y;
        }
        q += g.plane;
      }
    }
    __syncthreads();   // SE and the stage are free again
    if (tid == 0 && p + S <= p1_) issue(p + S, st, bars + stg);
    if (++stg == S) { stg = 0; par ^= 1u; }
  }
}

// ============================================================= adjoint ===
template <int TY, int S, int TW, int MODE>
__global__ void __launch_bounds__(TW / 2 * (TY + 2), (adj_ctas<S, MODE>()))
k_rev_adjoint(const __grid_constant__ RevMaps m, StepArgs a, RevUnits U) {
  typedef AL<TY, S, TW, MODE> Y;
  constexpr bool PXY = Y::PXY, PZ = Y::PZ;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * (TW / 2) + tx;
  int tix, tiy, cz;
  if (MODE == 2) {
    ring_unit(U, blockIdx.x, &tix, &tiy, &cz);
  } else {
    tix = blockIdx.x + a.t0x;
    tiy = blockIdx.y + a.t0y;
    cz = MODE == 1 ? zonly_chunk(U, blockIdx.z) : blockIdx.z + a.zc0;
  }
  const int x0 = tix * TW, y0 = tiy * TY;
  const int k0 = cz * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  // task: the tile's pair (main), a pair of the -y halo row, or a cell of the
  // -x halo column (as the second cell of a pair)
  const bool mainT = ty < TY;
  const bool rowT = ty == TY;
  const bool colT = ty == TY + 1 && tx < TY;
  const bool task = mainT || rowT || colT;
  const int x = colT ? x0 - 2 : x0 + 2 * tx;
  const int y = mainT ? y0 + ty : (rowT ? y0 - 1 : y0 + tx);
  const bool rowok = y >= 0 && y < g.ny;
  const bool ok0 = task && rowok && x >= 0 && x < g.nx;
  const bool ok1 = task && rowok && x + 1 >= 0 && x + 1 < g.nx;
  const bool v0 = mainT && ok0, v1 = mainT && ok1;   // cells this thread stores
  const int p0_ = k0 - 1, p1_ = k1;
  // ring units: the x / y CPML profiles the tile's cells and halo read,
  // staged once (they do not change along z), [6][TW+8] from x0-4 and
  // [6][TY+4] from y0-2
  float* SPX = reinterpret_cast<float*>(dsm + Y::SP);
  float* SPY = SPX + 6 * Y::SPXN;
  auto spx = [&](int w, int xx) { return SPX[w * Y::SPXN + xx - x0 + 4]; };
  auto spy = [&](int w, int yy) { return SPY[w * Y::SPYN + yy - y0 + 2]; };
  if (PXY) {
    const int nt = (TW / 2) * (TY + 2);
    for (int i = tid; i < 6 * Y::SPXN; i += nt) {
      const int w = i / Y::SPXN, xi = x0 - 4 + i % Y::SPXN;
      SPX[i] = (xi >= 0 && xi < g.nx) ? prof(g, 0, w, xi) : 0.f;
    }
    for (int i = tid; i < 6 * Y::SPYN; i += nt) {
      const int w = i / Y::SPYN, yi = y0 - 2 + i % Y::SPYN;
      SPY[i] = (yi >= 0 && yi < g.ny) ? prof(g, 1, w, yi) : 0.f;
    }
  }
  uint64_t* bars = ring_init<S>(dsm, Y::STAGE);   // at Y::BARS
  int qx0 = x0, qy0 = y0;
  bool txs = false, tys = false, txh = false, tyh = false;
  if (PXY) {
    psi_box_starts<TW, TY>(a.pl, x0, y0, &qx0, &qy0);
    txs = tile_in_slab(max(x0 - 2, 0), min(x0 + TW, g.nx - 1), g.nx, g.P);
    tys = tile_in_slab(max(y0 - 1, 0), min(y0 + TY, g.ny - 1), g.ny, g.P);
    txh = tile_in_slab(max(x0 - 1, 0), min(x0 + TW - 1, g.nx - 1), g.nx, g.P);
    tyh = tile_in_slab(max(y0 - 1, 0), min(y0 + TY - 1, g.ny - 1), g.ny, g.P);
  }
  auto inz = [&](int p) { return p >= 0 && p < g.nz; };
  auto boxes = [&](int p, auto&& f) {
    const bool tail = p == k1;
    if (!inz(p) && !(PZ && inz(p - 1) && p - 1 >= k0 - 1)) return;
    if (inz(p)) {
      f(Y::CB, &m.cb40, x0 - 4, y0 - 1, p, 0, Y::WP * 4);
      f(Y::LE, &m.L40, x0 - 4, y0 - 1, p, 0, 3 * Y::WP * 4);
      if (!tail) f(Y::LH, &m.L36, x0 - 4, y0 - 1, p, 3, 3 * Y::HP * 4);
    }
    const int pm = p - 1;
    if (PXY) {
      if (inz(p) && !tail && txs) f(Y::PEX, &m.Qx40, qx0 - 4, y0 - 1, p, 2, 2 * Y::EXP * 4);
      if (inz(p) && !tail && tys) f(Y::PEY, &m.Qy36, x0 - 4, qy0 - 1, p, 2, 2 * Y::EYP * 4);
      if (pm >= k0 && txh) f(Y::PHX, &m.Qxw, qx0 - 4, y0, pm, 0, 2 * Y::HXP * 4);
      if (pm >= k0 && tyh) f(Y::PHY, &m.Qyw, x0, qy0 - 1, pm, 0, 2 * Y::HYP * 4);
    }
    if (PZ) {
      if (inz(p) && in_slab(p, g.nz, g.P))
        f(Y::PEZ, &m.Qz36, x0 - 4, y0 - 1, psi_map(a.pl.ax[2], p), 2, 2 * Y::EZP * 4);
      if (pm >= k0 - 1 && inz(pm) && in_slab(pm, g.nz, g.P))
        f(Y::PHZ, &m.Qzo, x0, y0, psi_map(a.pl.ax[2], pm), 0, 2 * Y::HZP * 4);
    }
  };
  auto issue = [&](int p, unsigned char* st, uint64_t* bar) {
    stage_plane(boxes, p, st, bar, false);
  };
  if (tid == 0)
    for (int i = 0; i < S && p0_ + i <= p1_; ++i) issue(p0_ + i, dsm + i * Y::STAGE, bars + i);
  // x / y CPML profiles (ring units only): E side at x, x+1, x+2 and y, y+1; H side
  // at x-1, x, x+1 and y-1, y
  bool sx0 = false, sx1 = false, sx2 = false, sy = false, sy1 = false;
  bool hx0 = false, hx1 = false, hxm = false, hy = false, hym = false;
  if (PXY) {
    sx0 = ok0 && in_slab(x, g.nx, g.P);
    sx1 = ok1 && in_slab(x + 1, g.nx, g.P);
    sx2 = ok1 && x + 2 < g.nx && in_slab(x + 2, g.nx, g.P);
    sy = (ok0 || ok1) && in_slab(y, g.ny, g.P);
    sy1 = (ok0 || ok1) && y + 1 < g.ny && in_slab(y + 1, g.ny, g.P);
    hx0 = v0 && in_slab(x, g.nx, g.P);
    hx1 = v1 && in_slab(x + 1, g.nx, g.P);
    hxm = v0 && x > 0 && in_slab(x - 1, g.nx, g.P);
    hy = v0 && in_slab(y, g.ny, g.P);
    hym = v0 && y > 0 && in_slab(y - 1, g.ny, g.P);
  }
  const int wb = (y - y0 + 1) * Y::WW + (x - x0 + 4);   // the pair in the cb / lam_E boxes
  const int lb = (y - y0 + 1) * Y::HW + (x - x0 + 4);   // the pair in the lam_H box and SL
  float* SL = reinterpret_cast<float*>(dsm + Y::SL);
  const float S_ = g.S;
  const long long nc = g.nc;
  float* const Ln = a.Ln;
  float* const lpB = a.psiB;
  long long q = (long long)k0 * g.plane + (long long)y * g.px + x;   // plane k0 of the pair
  // lam_H'(p-1): own lam_H x, y, the +z terms pending and the completed x / y parts;
  // lam_Hz'(p-1) complete
  float c_lhx[2] = {0.f, 0.f}, c_lhy[2] = {0.f, 0.f}, c_o8[2] = {0.f, 0.f}, c_o7[2] = {0.f, 0.f};
  float c_bx[2] = {0.f, 0.f}, c_by[2] = {0.f, 0.f}, c_lhz[2] = {0.f, 0.f};
  // lam_E'(p-1): lam_E(p-1) and the -z terms of lam_H'(p-2)
  float c_le0[2] = {0.f, 0.f}, c_le1[2] = {0.f, 0.f}, c_le2[2] = {0.f, 0.f};
  float c_m1[2] = {0.f, 0.f}, c_m2[2] = {0.f, 0.f};
  int stg = 0;
  uint32_t par = 0;
  bool ok = true;
  for (int p = p0_; p <= p1_; ++p) {
    unsigned char* st = dsm + stg * Y::STAGE;
    if (!mbar_wait(bars + stg, par, kWaitCycles)) ok = false;
    if (!__syncthreads_and(ok)) { ring_abort<S>(bars, stg, par, p, p1_, a.err); return; }
    const float* CBb = reinterpret_cast<const float*>(st + Y::CB);
    const float* LEb = reinterpret_cast<const float*>(st + Y::LE);
    const float* LHb = reinterpret_cast<const float*>(st + Y::LH);
    const bool head = p < k0, tail = p == k1;
    const bool zs = PZ && inz(p) && in_slab(p, g.nz, g.P);
    float fx[2] = {0.f, 0.f}, fy[2] = {0.f, 0.f};   // lam_Hx', lam_Hy' of plane p-1
    float own_le[3][2];                              // lam_E(p) at the pair
    // ---- transpose of the E half-step: lam_H' ----
    if (task && (inz(p) || tail)) {
      if (!tail) {
        float o6[2], o11[2], o7[2], o8[2], o9[2], o10[2];
        float n6[2] = {0.f, 0.f}, n11[2] = {0.f, 0.f}, n9x = 0.f, n10x = 0.f;
        {
          const float2 cb2 = ld2(CBb, wb);
          const float2 lx2 = ld2(LEb, wb), ly2 = ld2(LEb + Y::WP, wb), lz2 = ld2(LEb + 2 * Y::WP, wb);
          own_le[0][0] = lx2.x; own_le[0][1] = lx2.y;
          own_le[1][0] = ly2.x; own_le[1][1] = ly2.y;
          own_le[2][0] = lz2.x; own_le[2][1] = lz2.y;
          const float cbv[2] = {cb2.x, cb2.y};
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const float wx = cbv[c] * own_le[0][c], wy = cbv[c] * own_le[1][c],
                        wz = cbv[c] * own_le[2][c];
            o6[c] = wx; o11[c] = -wz; o7[c] = -wx; o8[c] = wy; o9[c] = -wy; o10[c] = wz;
          }
          if (y + 1 < g.ny) {
            const float2 cy2 = ld2(CBb, wb + Y::WW);
            const float2 ly = ld2(LEb, wb + Y::WW), lz = ld2(LEb + 2 * Y::WP, wb + Y::WW);
            n6[0] = cy2.x * ly.x;
            n6[1] = cy2.y * ly.y;
            n11[0] = -cy2.x * lz.x;
            n11[1] = -cy2.y * lz.y;
          }
          if (x + 2 < g.nx) {
            const float c2 = CBb[wb + 2];
            n9x = -c2 * LEb[Y::WP + wb + 2];
            n10x = c2 * LEb[2 * Y::WP + wb + 2];
          }
        }
        if (PXY) {
          if (sy || sy1) {
            const float* P = reinterpret_cast<const float*>(st + Y::PEY);   // (TW+4) x (TY+2) at (x0-4, y0-1)
            const int yb = (y - y0 + 1) * (TW + 4) + (x - x0 + 4);
            if (sy) {
              const float by = spy(PR_BE, y), ay = spy(PR_AE, y), ky = spy(PR_KE, y);
              const float2 p0 = ld2(P, yb), p1 = ld2(P + Y::EYP, yb);
              const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
              float s6[2], s11[2];
#pragma unroll
              for (int c = 0; c < 2; ++c) {
                o6[c] = adj(o6[c], q0[c], by, ay, ky, &s6[c]);
                o11[c] = adj(o11[c], q1[c], by, ay, ky, &s11[c]);
              }
              if (!head && (v0 || v1)) {
                const long long qyy = psi_ix<1>(a.pl, 2, x, y, p);
                ST2(lpB, qyy, s6[0], s6[1], v0, v1);
                ST2(lpB + a.pl.ax[1].cs, qyy, s11[0], s11[1], v0, v1);
              }
            }
            if (sy1) {
              const float by1 = spy(PR_BE, y + 1), ay1 = spy(PR_AE, y + 1),
                          ky1 = spy(PR_KE, y + 1);
              const float2 p0 = ld2(P, yb + TW + 4), p1 = ld2(P + Y::EYP, yb + TW + 4);
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
            const float* P = reinterpret_cast<const float*>(st + Y::PEX);   // (TW+8) x (TY+1) at (x0-4, y0-1)
            const int xb = (y - y0 + 1) * (TW + 8) + (x - x0 + 4);
            const float2 p0 = ld2(P, xb), p1 = ld2(P + Y::EXP, xb);
            float s9[2] = {0.f, 0.f}, s10[2] = {0.f, 0.f};
            if (sx0) {
              const float b = spx(PR_BE, x), aa = spx(PR_AE, x), kk = spx(PR_KE, x);
              o9[0] = adj(o9[0], p0.x, b, aa, kk, &s9[0]);
              o10[0] = adj(o10[0], p1.x, b, aa, kk, &s10[0]);
            }
            if (sx1) {
              const float b = spx(PR_BE, x + 1), aa = spx(PR_AE, x + 1),
                          kk = spx(PR_KE, x + 1);
              o9[1] = adj(o9[1], p0.y, b, aa, kk, &s9[1]);
              o10[1] = adj(o10[1], p1.y, b, aa, kk, &s10[1]);
            }
            if (!head && ((v0 && sx0) || (v1 && sx1))) {
              const long long qxx = psi_ix<0>(a.pl, 2, x, y, p);
              ST2(lpB, qxx, s9[0], s9[1], v0 && sx0, v1 && sx1);
              ST2(lpB + a.pl.ax[0].cs, qxx, s10[0], s10[1], v0 && sx0, v1 && sx1);
            }
            if (sx2) {
              const float b = spx(PR_BE, x + 2), aa = spx(PR_AE, x + 2),
                          kk = spx(PR_KE, x + 2);
              float dummy;
              n9x = adj(n9x, P[xb + 2], b, aa, kk, &dummy);
              n10x = adj(n10x, P[Y::EXP + xb + 2], b, aa, kk, &dummy);
            }
          }
        }
        if (zs) {   // z-only and ring units
          const float* P = reinterpret_cast<const float*>(st + Y::PEZ);   // (TW+4) x (TY+1) at (x0-4, y0-1)
          const float b = prof(g, 2, PR_BE, p), aa = prof(g, 2, PR_AE, p), kv = prof(g, 2, PR_KE, p);
          const float2 p0 = ld2(P, lb), p1 = ld2(P + Y::EZP, lb);
          const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
          float s7[2], s8[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            o7[c] = adj(o7[c], q0[c], b, aa, kv, &s7[c]);
            o8[c] = adj(o8[c], q1[c], b, aa, kv, &s8[c]);
          }
          if (!head && (v0 || v1)) {
            const long long qz = psi_ix<2>(a.pl, 2, x, y, p);
            ST2(lpB, qz, s7[0], s7[1], v0, v1);
            ST2(lpB + a.pl.ax[2].cs, qz, s8[0], s8[1], v0, v1);
          }
        }
        // cell 0's +x terms are cell 1's own terms
        const float n9[2] = {ok1 ? o9[1] : 0.f, n9x}, n10[2] = {ok1 ? o10[1] : 0.f, n10x};
        const float2 lh0 = ld2(LHb, lb), lh1 = ld2(LHb + Y::HP, lb), lh2 = ld2(LHb + 2 * Y::HP, lb);
        if (!head) {   // finish lam_H'(p-1): its +z terms are this plane's o7, o8
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            fx[c] = c_lhx[c] + ((c_o8[c] - o8[c]) + c_bx[c]);
            fy[c] = c_lhy[c] + ((c_o7[c] - o7[c]) + c_by[c]);
          }
        }
        const float lhz[2] = {lh2.x + ((o6[0] - n6[0]) + (o9[0] - n9[0])),
                              lh2.y + ((o6[1] - n6[1]) + (o9[1] - n9[1]))};
        if (!head) {
          *reinterpret_cast<float2*>(SL + lb) = make_float2(fx[0], fx[1]);
          *reinterpret_cast<float2*>(SL + Y::HP + lb) = make_float2(fy[0], fy[1]);
          *reinterpret_cast<float2*>(SL + 2 * Y::HP + lb) = make_float2(c_lhz[0], c_lhz[1]);
          if (p - 1 >= k0) {
            const long long qm = q - g.plane;
            ST2(Ln + 3 * nc, qm, fx[0], fx[1], v0, v1);
            ST2(Ln + 4 * nc, qm, fy[0], fy[1], v0, v1);
            ST2(Ln + 5 * nc, qm, c_lhz[0], c_lhz[1], v0, v1);
          }
        }
        c_lhx[0] = lh0.x; c_lhx[1] = lh0.y;
        c_lhy[0] = lh1.x; c_lhy[1] = lh1.y;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          c_lhz[c] = lhz[c];
          c_o8[c] = o8[c];
          c_o7[c] = o7[c];
          c_bx[c] = o11[c] - n11[c];
          c_by[c] = o10[c] - n10[c];
        }
      } else {   // tail: finish lam_H'(k1-1) with the +z terms of plane k1
        float n7[2] = {0.f, 0.f}, n8[2] = {0.f, 0.f};
        if (inz(p)) {
          const float2 c2 = ld2(CBb, wb), lx = ld2(LEb, wb), ly = ld2(LEb + Y::WP, wb);
          n7[0] = -c2.x * lx.x;
          n7[1] = -c2.y * lx.y;
          n8[0] = c2.x * ly.x;
          n8[1] = c2.y * ly.y;
          if (zs) {
            const float* P = reinterpret_cast<const float*>(st + Y::PEZ);
            const float b1 = prof(g, 2, PR_BE, p), a1 = prof(g, 2, PR_AE, p), k1v = prof(g, 2, PR_KE, p);
            const float2 p0 = ld2(P, lb), p1 = ld2(P + Y::EZP, lb);
            const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
            float dummy;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              n7[c] = adj(n7[c], q0[c], b1, a1, k1v, &dummy);
              n8[c] = adj(n8[c], q1[c], b1, a1, k1v, &dummy);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          fx[c] = c_lhx[c] + ((c_o8[c] - n8[c]) + c_bx[c]);
          fy[c] = c_lhy[c] + ((c_o7[c] - n7[c]) + c_by[c]);
        }
        *reinterpret_cast<float2*>(SL + lb) = make_float2(fx[0], fx[1]);
        *reinterpret_cast<float2*>(SL + Y::HP + lb) = make_float2(fy[0], fy[1]);
        *reinterpret_cast<float2*>(SL + 2 * Y::HP + lb) = make_float2(c_lhz[0], c_lhz[1]);
        const long long qm = q - g.plane;
        ST2(Ln + 3 * nc, qm, fx[0], fx[1], v0, v1);
        ST2(Ln + 4 * nc, qm, fy[0], fy[1], v0, v1);
        ST2(Ln + 5 * nc, qm, c_lhz[0], c_lhz[1], v0, v1);
      }
    }
    __syncthreads();   // lam_H'(p-1) of the tile and its halo is in SL
    // ---- transpose of the H half-step, one plane behind: lam_E'(p-1) ----
    if (mainT && !head) {
      if (p - 1 >= k0) {
        const float2 lx2 = ld2(SL, lb), ly2 = ld2(SL + Y::HP, lb), lz2 = ld2(SL + 2 * Y::HP, lb);
        float o0[2], o1[2], o2[2], o3[2], o4[2], o5[2];
        {
          const float lhx[2] = {lx2.x, lx2.y}, lhy[2] = {ly2.x, ly2.y}, lhz[2] = {lz2.x, lz2.y};
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            o0[c] = -S_ * lhx[c];
            o5[c] = S_ * lhz[c];
            o1[c] = S_ * lhx[c];
            o2[c] = -S_ * lhy[c];
            o3[c] = S_ * lhy[c];
            o4[c] = -S_ * lhz[c];
          }
        }
        float m0[2], m5[2];
        {
          const float2 lxy = ld2(SL, lb - Y::HW), lzy = ld2(SL + 2 * Y::HP, lb - Y::HW);   // -y
          m0[0] = -S_ * lxy.x; m0[1] = -S_ * lxy.y;
          m5[0] = S_ * lzy.x;  m5[1] = S_ * lzy.y;
        }
        float m3x = S_ * SL[Y::HP + lb - 1], m4x = -S_ * SL[2 * Y::HP + lb - 1];   // -x of cell 0
        if (y == 0) { m0[0] = 0.f; m0[1] = 0.f; m5[0] = 0.f; m5[1] = 0.f; }
        if (x == 0) { m3x = 0.f; m4x = 0.f; }
        const int pm = p - 1;
        {
          if (PXY && (hy || hym)) {
            const float* P = reinterpret_cast<const float*>(st + Y::PHY);   // TW x (TY+1) at (x0, y0-1)
            const int yb = (y - y0 + 1) * TW + (x - x0);
            if (hy) {
              const float by = spy(PR_BH, y), ay = spy(PR_AH, y), ky = spy(PR_KH, y);
              const float2 p0 = ld2(P, yb), p1 = ld2(P + Y::HYP, yb);
              const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
              float s4[2], s5[2];
#pragma unroll
              for (int c = 0; c < 2; ++c) {
                o0[c] = adj(o0[c], q0[c], by, ay, ky, &s4[c]);
                o5[c] = adj(o5[c], q1[c], by, ay, ky, &s5[c]);
              }
              const long long qyy = psi_ix<1>(a.pl, 0, x, y, pm);
              ST2(lpB, qyy, s4[0], s4[1], v0, v1);
              ST2(lpB + a.pl.ax[1].cs, qyy, s5[0], s5[1], v0, v1);
            }
            if (hym) {
              const float bym = spy(PR_BH, y - 1), aym = spy(PR_AH, y - 1),
                          kym = spy(PR_KH, y - 1);
              const float2 p0 = ld2(P, yb - TW), p1 = ld2(P + Y::HYP, yb - TW);
              const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
              float dummy;
#pragma unroll
              for (int c = 0; c < 2; ++c) {
                m0[c] = adj(m0[c], q0[c], bym, aym, kym, &dummy);
                m5[c] = adj(m5[c], q1[c], bym, aym, kym, &dummy);
              }
            }
          }
          if (PXY && (hx0 || hx1 || hxm)) {
            const float* P = reinterpret_cast<const float*>(st + Y::PHX);   // (TW+4) x TY at (x0-4, y0)
            const int xb = (y - y0) * (TW + 4) + (x - x0 + 4);
            const float2 p0 = ld2(P, xb), p1 = ld2(P + Y::HXP, xb);
            float s0[2] = {0.f, 0.f}, s1[2] = {0.f, 0.f};
            if (hx0) {
              const float b = spx(PR_BH, x), aa = spx(PR_AH, x), kk = spx(PR_KH, x);
              o3[0] = adj(o3[0], p0.x, b, aa, kk, &s0[0]);
              o4[0] = adj(o4[0], p1.x, b, aa, kk, &s1[0]);
            }
            if (hx1) {
              const float b = spx(PR_BH, x + 1), aa = spx(PR_AH, x + 1),
                          kk = spx(PR_KH, x + 1);
              o3[1] = adj(o3[1], p0.y, b, aa, kk, &s0[1]);
              o4[1] = adj(o4[1], p1.y, b, aa, kk, &s1[1]);
            }
            const long long qxx = psi_ix<0>(a.pl, 0, x, y, pm);
            ST2(lpB, qxx, s0[0], s0[1], hx0, hx1);
            ST2(lpB + a.pl.ax[0].cs, qxx, s1[0], s1[1], hx0, hx1);
            if (hxm) {
              const float b = spx(PR_BH, x - 1), aa = spx(PR_AH, x - 1),
                          kk = spx(PR_KH, x - 1);
              float dummy;
              m3x = adj(m3x, P[xb - 1], b, aa, kk, &dummy);
              m4x = adj(m4x, P[Y::HXP + xb - 1], b, aa, kk, &dummy);
            }
          }
          if (PZ && in_slab(pm, g.nz, g.P)) {
            const float* P = reinterpret_cast<const float*>(st + Y::PHZ);   // TW x TY at (x0, y0)
            const int zb = (y - y0) * TW + (x - x0);
            const float b = prof(g, 2, PR_BH, pm), aa = prof(g, 2, PR_AH, pm), kv = prof(g, 2, PR_KH, pm);
            const float2 p0 = ld2(P, zb), p1 = ld2(P + Y::HZP, zb);
            const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
            float s8[2], s9[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              o1[c] = adj(o1[c], q0[c], b, aa, kv, &s8[c]);
              o2[c] = adj(o2[c], q1[c], b, aa, kv, &s9[c]);
            }
            const long long qz = psi_ix<2>(a.pl, 0, x, y, pm);
            ST2(lpB, qz, s8[0], s8[1], v0, v1);
            ST2(lpB + a.pl.ax[2].cs, qz, s9[0], s9[1], v0, v1);
          }
        }
        // cell 1's -x terms are cell 0's own terms
        const float m3[2] = {m3x, o3[0]}, m4[2] = {m4x, o4[0]};
        const long long qm = q - g.plane;
        ST2(Ln, qm, c_le0[0] + ((c_m2[0] - o2[0]) + (m5[0] - o5[0])),
            c_le0[1] + ((c_m2[1] - o2[1]) + (m5[1] - o5[1])), v0, v1);
        ST2(Ln + nc, qm, c_le1[0] + ((c_m1[0] - o1[0]) + (m4[0] - o4[0])),
            c_le1[1] + ((c_m1[1] - o1[1]) + (m4[1] - o4[1])), v0, v1);
        ST2(Ln + 2 * nc, qm, c_le2[0] + ((m0[0] - o0[0]) + (m3[0] - o3[0])),
            c_le2[1] + ((m0[1] - o0[1]) + (m3[1] - o3[1])), v0, v1);
        // the -z terms plane p needs are this plane's own z-terms
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          c_m1[c] = o1[c];
          c_m2[c] = o2[c];
        }
      } else {   // p == k0: the own z-terms of lam_H'(k0-1) for lam_E'(k0)
        float m1n[2] = {0.f, 0.f}, m2n[2] = {0.f, 0.f};
        const int pm = p - 1;
        if (pm >= 0) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            m1n[c] = S_ * fx[c];
            m2n[c] = -S_ * fy[c];
          }
          if (PZ && in_slab(pm, g.nz, g.P)) {
            const float* P = reinterpret_cast<const float*>(st + Y::PHZ);
            const int zb = (y - y0) * TW + (x - x0);
            const float b1 = prof(g, 2, PR_BH, pm), a1 = prof(g, 2, PR_AH, pm), k1v = prof(g, 2, PR_KH, pm);
            const float2 p0 = ld2(P, zb), p1 = ld2(P + Y::HZP, zb);
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
    if (mainT && !tail) {   // lam_E(p) at the pair, for lam_E'(p) one plane later
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        c_le0[c] = own_le[0][c];
        c_le1[c] = own_le[1][c];
        c_le2[c] = own_le[2][c];
      }
      if (!head) q += g.plane;
    }
    __syncthreads();   // SL and the stage are free again
    if (tid == 0 && p + S <= p1_) issue(p + S, st, bars + stg);
    if (++stg == S) { stg = 0; par ^= 1u; }
  }
}

// ------------------------------------------------------------ launchers ---
template <class KT, class... Args>
static cudaError_t launch_rf(KT kernel, dim3 grid, dim3 block, int smem, cudaStream_t s,
                             Args... args) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e) return e;
  kernel<<<grid, block, smem, s>>>(args...);
  return cudaGetLastError();
}

template <int TY>
static cudaError_t launch_rev_fused_t(int which, const RevMaps& m, const StepArgs& a,
                                      const RevUnits& U, dim3 grid, cudaStream_t s) {
  constexpr int TW = 32;
  const dim3 block(TW / 2, TY + 2);
  switch (which) {
    case 0:
      if (a.xq)
        return launch_rf(k_rev_primal<TY, 3, TW, true>, grid, block, PL<TY, 3, TW>::smem(), s, m, a);
      return launch_rf(k_rev_primal<TY, 3, TW, false>, grid, block, PL<TY, 3, TW>::smem(), s, m, a);
    case 1:
      return launch_rf(k_rev_adjoint<TY, 3, TW, 0>, grid, block, AL<TY, 3, TW, 0>::smem(), s, m, a, U);
    case 2:
      return launch_rf(k_rev_adjoint<TY, 3, TW, 1>, grid, block, AL<TY, 3, TW, 1>::smem(), s, m, a, U);
    case 3:
      return launch_rf(k_rev_adjoint<TY, 2, TW, 2>, grid, block, AL<TY, 2, TW, 2>::smem(), s, m, a, U);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_rev_fused(int which, const RevMaps& m, const StepArgs& a, const RevUnits& U,
                             cudaStream_t s) {
  const int TW = 32, TY = 8;
  if (a.tile_y != TY || a.tile_x != TW) return cudaErrorInvalidValue;
  dim3 grid(0, 0, 0);
  StepArgs b = a;
  const int nzin = U.iz1 - U.iz0;
  switch (which) {
    case 0:
      grid = dim3(U.px1 - U.px0, U.py1 - U.py0, U.pz1 - U.pz0);
      b.t0x = U.px0; b.t0y = U.py0; b.zc0 = U.pz0;
      break;
    case 1:
      grid = dim3(U.ix1 - U.ix0, U.iy1 - U.iy0, nzin);
      b.t0x = U.ix0; b.t0y = U.iy0; b.zc0 = U.iz0;
      break;
    case 2:
      grid = dim3(U.ix1 - U.ix0, U.iy1 - U.iy0, U.nzc - nzin);
      b.t0x = U.ix0; b.t0y = U.iy0; b.zc0 = 0;
      break;
    case 3:
      grid = dim3((unsigned)(ring_tiles(U) * U.nzc), 1, 1);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
  return launch_rev_fused_t<8>(which, m, b, U, grid, s);
}

// Tiles and chunks of the three launches (host and tests).
RevUnits rev_units(const Geo& g, int zchunk) {
  const int TW = 32, TY = 8;
  RevUnits U = {};
  const int P = g.P, zc = zchunk > 0 ? zchunk : g.nz;
  U.ntx = (g.nx + TW - 1) / TW;
  U.nty = (g.ny + TY - 1) / TY;
  U.nzc = (g.nz + zc - 1) / zc;
  // primal: every tile and chunk with an interior cell
  U.px0 = P / TW; U.px1 = (g.nx - P - 1) / TW + 1;
  U.py0 = P / TY; U.py1 = (g.ny - P - 1) / TY + 1;
  U.pz0 = P / zc; U.pz1 = (g.nz - P - 1) / zc + 1;
  if (g.nx - 2 * P <= 0 || g.ny - 2 * P <= 0 || g.nz - 2 * P <= 0) {
    U.px0 = U.px1 = U.py0 = U.py1 = U.pz0 = U.pz1 = 0;
  }
  // adjoint without CPML terms: every cell the CTA evaluates a term of lies
  // in the interior, x in [x0-1, x0+TW], y in [y0-1, y0+TY], z in [k0-1, k1]
  auto lo = [](int need, int t) { return (need + t - 1) / t; };   // first tile with t0 >= need
  U.ix0 = lo(P + 1, TW);
  U.ix1 = (g.nx - P - 1 - TW) >= 0 ? (g.nx - P - 1 - TW) / TW + 1 : 0;
  U.iy0 = lo(P + 1, TY);
  U.iy1 = (g.ny - P - 1 - TY) >= 0 ? (g.ny - P - 1 - TY) / TY + 1 : 0;
  U.iz0 = lo(P + 1, zc);
  U.iz1 = (g.nz - P - 1 - zc) >= 0 ? (g.nz - P - 1 - zc) / zc + 1 : 0;
  // the last chunk may be short: k1 = min(nz, k0 + zc) <= nz - P - 1 holds for
  // every chunk below iz1 since those are full chunks
  if (U.ix1 <= U.ix0 || U.iy1 <= U.iy0 || U.iz1 <= U.iz0) {
    U.ix0 = U.ix1 = U.iy0 = U.iy1 = U.iz0 = U.iz1 = 0;
  }
  return U;
}

void rev_zonly_unit(const RevUnits& U, int bx, int by, int bz, int* tx, int* ty, int* cz) {
  *tx = bx + U.ix0;
  *ty = by + U.iy0;
  *cz = zonly_chunk(U, bz);
}

void rev_ring_unit(const RevUnits& U, long long u, int* tx, int* ty, int* cz) {
  ring_unit(U, u, tx, ty, cz);
}

long long rev_ring_tiles(const RevUnits& U) { return ring_tiles(U); }

}  // namespace fdtd
