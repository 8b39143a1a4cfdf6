// kernels_fwd_2step.cu -- two forward time steps of the deep interior in one pass
// (temporal blocking of the leapfrog whose gradient Sec. 2 computes).
//
// Steps n and n + 1:
//     Ht1 = Ht^{n+1/2} = Ht^{n-1/2} - S curl E^n      (forward differences)
//     E1  = E^{n+1}    = E^n + cb curl Ht1            (backward differences)
//     Ht2 = Ht^{n+3/2} = Ht1 - S curl E1
//     E2  = E^{n+2}    = E1 + cb curl Ht2
// A CTA reads E^n, Ht^{n-1/2} and cb of its unit once and writes E2 and Ht2
// once (52 B per cell for two time steps, against 104 B for two fused
// steps).  The intermediate level exists only in shared memory, on halos
// that shrink by one cell per half-step: E2 on the 32 x 8 tile T needs Ht2
// on T and its -x / -y neighbours (R1), Ht2 on R1 needs E1 on R1 and its
// +x / +y neighbours (R2), E1 on R2 needs Ht1 on R2 and its -x / -y
// neighbours (R3), and Ht1 on R3 needs E^n on R3 and its +x / +y neighbours
// (R4).  One thread per pair of x cells on R3: 18 pair columns (x = x0 - 2 +
// 2 px) by 11 rows (y = y0 - 2 + ry); R2 is rows ry >= 1, R1 rows 1..9 and
// pair columns 0..16, T rows 2..9 and pair columns 1..16.  Along z the
// levels lag one plane each: with E^n of plane p staged, the CTA finishes
// Ht1(p - 1), updates E1(p - 1), then Ht2(p - 2) and E2(p - 2); a chunk
// [k0, k1) streams the planes k0 - 2 .. k1 + 1.
//
// The launch covers the deep units: every cell on which the CTA evaluates a
// level (R3 over the planes k0 - 2 .. k1) lies in the interior, so no CPML
// term arises, and the host keeps the source and the detectors away from
// them.  The other units run the split half-steps one time step at a time,
// through a third buffer Fm that holds the intermediate level: they need
// E1 and Ht1 only on the deep units' cells next to their own, i.e. on the
// one-cell frame of the deep box, which this kernel writes into Fm.  Every
// cell sees the same explicitly rounded operations as in the split and the
// fused kernels, so the fields are bit-identical to theirs.
#include <cudaTypedefs.h>

#include "lag_common.cuh"

namespace fdtd {

using namespace lag2;

namespace fwd2s {

constexpr int TW = 32, TY = 8;
constexpr int NPX = 18, NRY = 11, NT = NPX * NRY;   // pair tasks of R3
constexpr int THREADS = 224;                        // 7 warps
constexpr int BW = 40;                              // row width: x in [x0 - 4, x0 + 36)

// Shared memory (byte offsets): S stages of an E^n box and an Ht^{n-1/2}
// box, 40 x 12 at (x0 - 4, y0 - 2), 3 components each, and a cb box 40 x 10
// at (x0 - 4, y0 - 1); the stages' mbarriers after them; then Ht1 of one
// plane, E1 of two planes (ping-pong by plane parity) and Ht2 of one plane,
// each [3][11][40] at (x0 - 4, y0 - 2).
template <int S>
struct L2S {
  static constexpr int BP = BW * 12;    // one component of a staged field box
  static constexpr int CBP = BW * 10;   // the cb box
  static constexpr int AP = BW * NRY;   // one component of a level's plane array
  static constexpr int E = 0;
  static constexpr int H = E + r128(3 * BP * 4);
  static constexpr int CB = H + r128(3 * BP * 4);
  static constexpr int STAGE = CB + r128(CBP * 4);
  static constexpr int BARS = S * STAGE;
  static constexpr int H1 = r128(BARS + 8 * S);
  static constexpr int E1 = H1 + r128(3 * AP * 4);
  static constexpr int H2 = E1 + 2 * r128(3 * AP * 4);
  static int smem() { return H2 + 3 * AP * 4; }
};

static_assert(L2S<3>::H1 >= L2S<3>::BARS + 8 * 3, "level arrays after the barriers");
static_assert(NT <= THREADS, "one pair task per thread");

template <int S, bool EX>
__global__ void __launch_bounds__(THREADS, 3)
k_fwd_2step(const __grid_constant__ Fwd2Maps m, StepArgs a) {
  typedef L2S<S> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tid = threadIdx.x;
  const int x0 = (blockIdx.x + a.U.ix0) * TW, y0 = (blockIdx.y + a.U.iy0) * TY;
  // the deep box in cells, and this CTA's chunk of it
  const int X0 = a.U.ix0 * TW, X1 = a.U.ix1 * TW, Y0 = a.U.iy0 * TY, Y1 = a.U.iy1 * TY;
  const int Z0 = a.U.iz0 * a.zcs, Z1 = min(g.nz, a.U.iz1 * a.zcs);
  const int k0 = Z0 + blockIdx.z * a.zchunk, k1 = min(Z1, k0 + a.zchunk);
  const bool task = tid < NT;
  const int px = task ? tid % NPX : 0, ry = task ? tid / NPX : 0;
  const int x = x0 - 2 + 2 * px, y = y0 - 2 + ry;
  const bool r2 = task && ry >= 1;                         // R2
  const bool r1 = r2 && ry <= 9 && px <= 16;               // R1
  const bool tt = r1 && ry >= 2 && px >= 1;                // T
  const int hb = ry * BW + (x - x0 + 4);                   // the pair in a box or level array
  const int cbi = (ry - 1) * BW + (x - x0 + 4);            // the pair in the cb box (R2)
  // frame cells of the deep box (the intermediate level goes to Fm there)
  const bool fxy0 = y == Y0 || y == Y1 - 1 || x == X0;
  const bool fxy1 = y == Y0 || y == Y1 - 1 || x + 1 == X1 - 1;
  const int p0_ = k0 - 2, p1_ = k1 + 1;
  uint64_t* bars = ring_init<S>(dsm, Y::STAGE);   // at Y::BARS
  auto boxes = [&](int p, auto&& f) {
    f(Y::E, &m.F4012, x0 - 4, y0 - 2, p, 0, 3 * Y::BP * 4);
    if (p <= k1) f(Y::H, &m.F4012, x0 - 4, y0 - 2, p, 3, 3 * Y::BP * 4);
    if (p >= k0 - 1 && p <= k1) f(Y::CB, &m.cb40, x0 - 4, y0 - 1, p, 0, Y::CBP * 4);
  };
  auto issue = [&](int p, unsigned char* st, uint64_t* bar) {
    stage_plane(boxes, p, st, bar, false);
  };
  if (tid == 0)
    for (int i = 0; i < S && p0_ + i <= p1_; ++i) issue(p0_ + i, dsm + i * Y::STAGE, bars + i);
  float* SH1 = reinterpret_cast<float*>(dsm + Y::H1);
  float* SE1 = reinterpret_cast<float*>(dsm + Y::E1);
  float* SH2 = reinterpret_cast<float*>(dsm + Y::H2);
  constexpr int AP = Y::AP, SE1P = r128(3 * AP * 4) / 4;   // floats per E1 plane array
  const float S_ = g.S;
  const long long nc = g.nc;
  float* const Fn = a.Fn;
  float* const Fm = a.Fm;
  const long long qxy = (long long)y * g.px + x;
  // Ht1(p) in progress (set when plane p is staged): E^n(p) at the pair, the
  // x / y difference terms, Ht^{n-1/2}(p)
  float c_ex[2] = {0.f, 0.f}, c_ey[2] = {0.f, 0.f}, c_ez[2] = {0.f, 0.f};
  float c_t0[2] = {0.f, 0.f}, c_t3[2] = {0.f, 0.f}, c_t4[2] = {0.f, 0.f}, c_t5[2] = {0.f, 0.f};
  float c_hx[2] = {0.f, 0.f}, c_hy[2] = {0.f, 0.f}, c_hz[2] = {0.f, 0.f};
  // carried levels at the pair: cb(p - 1), cb(p - 2), Ht1(p - 2), E1(p - 2),
  // Ht2(p - 3) x / y
  float c_cb1[2] = {0.f, 0.f}, c_cb2[2] = {0.f, 0.f};
  float c_h1x[2] = {0.f, 0.f}, c_h1y[2] = {0.f, 0.f}, c_h1z[2] = {0.f, 0.f};
  float c_e1x[2] = {0.f, 0.f}, c_e1y[2] = {0.f, 0.f}, c_e1z[2] = {0.f, 0.f};
  float c_h2x[2] = {0.f, 0.f}, c_h2y[2] = {0.f, 0.f};
  int stg = 0;
  uint32_t par = 0;
  bool ok = true;
  for (int p = p0_; p <= p1_; ++p) {
    unsigned char* st = dsm + stg * Y::STAGE;
    if (!mbar_wait(bars + stg, par, kWaitCycles)) ok = false;
    if (!__syncthreads_and(ok)) { ring_abort<S>(bars, stg, par, p, p1_, a.err); return; }
    const float* Eb = reinterpret_cast<const float*>(st + Y::E);
    // ---- A: finish Ht1(p - 1) with dEy/dz and dEx/dz ----
    float fx[2] = {0.f, 0.f}, fy[2] = {0.f, 0.f}, fz[2] = {0.f, 0.f};
    if (task && p >= k0 - 1) {
      const float2 ex2 = ld2(Eb, hb), ey2 = ld2(Eb + Y::BP, hb);
      const float ex[2] = {ex2.x, ex2.y}, ey[2] = {ey2.x, ey2.y};
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float t1 = ey[c] - c_ey[c], t2 = ex[c] - c_ex[c];
        const float cx = c_t0[c] - t1, cy = t2 - c_t3[c], cz = c_t4[c] - c_t5[c];
        fx[c] = __fsub_rn(c_hx[c], inc_of<EX>(__fmul_rn(S_, cx), a));
        fy[c] = __fsub_rn(c_hy[c], inc_of<EX>(__fmul_rn(S_, cy), a));
        fz[c] = __fsub_rn(c_hz[c], inc_of<EX>(__fmul_rn(S_, cz), a));
      }
      *reinterpret_cast<float2*>(SH1 + hb) = make_float2(fx[0], fx[1]);
      *reinterpret_cast<float2*>(SH1 + AP + hb) = make_float2(fy[0], fy[1]);
      *reinterpret_cast<float2*>(SH1 + 2 * AP + hb) = make_float2(fz[0], fz[1]);
      const int z = p - 1;
      if (tt && z >= k0 && z < k1) {
        const bool fz_ = z == Z0 || z == Z1 - 1;
        const bool f0 = fz_ || fxy0, f1 = fz_ || fxy1;
        if (f0 || f1) {
          const long long q = (long long)z * g.plane + qxy;
          ST2(Fm + 3 * nc, q, fx[0], fx[1], f0, f1);
          ST2(Fm + 4 * nc, q, fy[0], fy[1], f0, f1);
          ST2(Fm + 5 * nc, q, fz[0], fz[1], f0, f1);
        }
      }
    }
    __syncthreads();   // Ht1(p - 1) of R3 is in SH1
    // ---- B1: E1(p - 1) on R2 ----
    float ux[2] = {0.f, 0.f}, uy[2] = {0.f, 0.f}, uz[2] = {0.f, 0.f};   // E1(p - 1)
    const bool b1 = r2 && p >= k0 && p <= k1 + 1;
    if (b1) {
      const float2 hzy = ld2(SH1 + 2 * AP, hb - BW), hxy = ld2(SH1, hb - BW);   // -y
      const float hzx = SH1[2 * AP + hb - 1], hyx = SH1[AP + hb - 1];             // -x of cell 0
      const float d6[2] = {fz[0] - hzy.x, fz[1] - hzy.y};          // dHz/dy
      const float d7[2] = {fy[0] - c_h1y[0], fy[1] - c_h1y[1]};    // dHy/dz
      const float d8[2] = {fx[0] - c_h1x[0], fx[1] - c_h1x[1]};    // dHx/dz
      const float d9[2] = {fz[0] - hzx, fz[1] - fz[0]};            // dHz/dx
      const float d10[2] = {fy[0] - hyx, fy[1] - fy[0]};           // dHy/dx
      const float d11[2] = {fx[0] - hxy.x, fx[1] - hxy.y};         // dHx/dy
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float c0 = d6[c] - d7[c], c1 = d8[c] - d9[c], c2 = d10[c] - d11[c];
        ux[c] = __fadd_rn(c_ex[c], inc_of<EX>(__fmul_rn(c_cb1[c], c0), a));
        uy[c] = __fadd_rn(c_ey[c], inc_of<EX>(__fmul_rn(c_cb1[c], c1), a));
        uz[c] = __fadd_rn(c_ez[c], inc_of<EX>(__fmul_rn(c_cb1[c], c2), a));
      }
      float* E1w = SE1 + ((p - 1) & 1) * SE1P;
      *reinterpret_cast<float2*>(E1w + hb) = make_float2(ux[0], ux[1]);
      *reinterpret_cast<float2*>(E1w + AP + hb) = make_float2(uy[0], uy[1]);
      *reinterpret_cast<float2*>(E1w + 2 * AP + hb) = make_float2(uz[0], uz[1]);
      const int z = p - 1;
      if (tt && z >= k0 && z < k1) {
        const bool fz_ = z == Z0 || z == Z1 - 1;
        const bool f0 = fz_ || fxy0, f1 = fz_ || fxy1;
        if (f0 || f1) {
          const long long q = (long long)z * g.plane + qxy;
          ST2(Fm, q, ux[0], ux[1], f0, f1);
          ST2(Fm + nc, q, uy[0], uy[1], f0, f1);
          ST2(Fm + 2 * nc, q, uz[0], uz[1], f0, f1);
        }
      }
    }
    // ---- B2: Ht2(p - 2) on R1, from E1(p - 2) (SE1) and E1(p - 1) ----
    float gx[2] = {0.f, 0.f}, gy[2] = {0.f, 0.f}, gz[2] = {0.f, 0.f};   // Ht2(p - 2)
    if (r1 && p >= k0 + 1 && p <= k1 + 1) {
      const float* E1r = SE1 + (p & 1) * SE1P;   // plane p - 2
      const float2 ex2 = ld2(E1r, hb), ey2 = ld2(E1r + AP, hb), ez2 = ld2(E1r + 2 * AP, hb);
      const float2 ezy = ld2(E1r + 2 * AP, hb + BW), exy = ld2(E1r, hb + BW);   // +y
      const float ezx = E1r[2 * AP + hb + 2], eyx = E1r[AP + hb + 2];           // +x of cell 1
      const float t0[2] = {ezy.x - ez2.x, ezy.y - ez2.y};   // dEz/dy
      const float t3[2] = {ez2.y - ez2.x, ezx - ez2.y};     // dEz/dx
      const float t4[2] = {ey2.y - ey2.x, eyx - ey2.y};     // dEy/dx
      const float t5[2] = {exy.x - ex2.x, exy.y - ex2.y};   // dEx/dy
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float t1 = uy[c] - c_e1y[c], t2 = ux[c] - c_e1x[c];
        const float cx = t0[c] - t1, cy = t2 - t3[c], cz = t4[c] - t5[c];
        gx[c] = __fsub_rn(c_h1x[c], inc_of<EX>(__fmul_rn(S_, cx), a));
        gy[c] = __fsub_rn(c_h1y[c], inc_of<EX>(__fmul_rn(S_, cy), a));
        gz[c] = __fsub_rn(c_h1z[c], inc_of<EX>(__fmul_rn(S_, cz), a));
      }
      *reinterpret_cast<float2*>(SH2 + hb) = make_float2(gx[0], gx[1]);
      *reinterpret_cast<float2*>(SH2 + AP + hb) = make_float2(gy[0], gy[1]);
      *reinterpret_cast<float2*>(SH2 + 2 * AP + hb) = make_float2(gz[0], gz[1]);
      const int z = p - 2;
      if (tt && z >= k0 && z < k1) {
        const long long q = (long long)z * g.plane + qxy;
        ST2(Fn + 3 * nc, q, gx[0], gx[1], true, true);
        ST2(Fn + 4 * nc, q, gy[0], gy[1], true, true);
        ST2(Fn + 5 * nc, q, gz[0], gz[1], true, true);
      }
    }
    // ---- B3: start Ht1(p): its x and y differences ----
    float n_cb[2] = {0.f, 0.f};
    if (task && p <= k1) {
      const float2 ex2 = ld2(Eb, hb), ey2 = ld2(Eb + Y::BP, hb), ez2 = ld2(Eb + 2 * Y::BP, hb);
      const float2 ezy = ld2(Eb + 2 * Y::BP, hb + BW), exy = ld2(Eb, hb + BW);   // +y
      const float ezx = Eb[2 * Y::BP + hb + 2], eyx = Eb[Y::BP + hb + 2];         // +x of cell 1
      const float* Hb = reinterpret_cast<const float*>(st + Y::H);
      const float2 h0 = ld2(Hb, hb), h1 = ld2(Hb + Y::BP, hb), h2 = ld2(Hb + 2 * Y::BP, hb);
      c_t0[0] = ezy.x - ez2.x; c_t0[1] = ezy.y - ez2.y;   // dEz/dy
      c_t3[0] = ez2.y - ez2.x; c_t3[1] = ezx - ez2.y;     // dEz/dx
      c_t4[0] = ey2.y - ey2.x; c_t4[1] = eyx - ey2.y;     // dEy/dx
      c_t5[0] = exy.x - ex2.x; c_t5[1] = exy.y - ex2.y;   // dEx/dy
      c_ex[0] = ex2.x; c_ex[1] = ex2.y;
      c_ey[0] = ey2.x; c_ey[1] = ey2.y;
      c_ez[0] = ez2.x; c_ez[1] = ez2.y;
      c_hx[0] = h0.x; c_hx[1] = h0.y;
      c_hy[0] = h1.x; c_hy[1] = h1.y;
      c_hz[0] = h2.x; c_hz[1] = h2.y;
      if (r2 && p >= k0 - 1) {
        const float2 cb2 = ld2(reinterpret_cast<const float*>(st + Y::CB), cbi);
        n_cb[0] = cb2.x; n_cb[1] = cb2.y;
      }
    }
    __syncthreads();   // Ht2(p - 2) of R1 is in SH2; the stage is free again
    if (tid == 0 && p + S <= p1_) issue(p + S, st, bars + stg);
    // ---- C: E2(p - 2) on T ----
    if (tt && p >= k0 + 2) {
      const float2 hzy = ld2(SH2 + 2 * AP, hb - BW), hxy = ld2(SH2, hb - BW);   // -y
      const float hzx = SH2[2 * AP + hb - 1], hyx = SH2[AP + hb - 1];             // -x of cell 0
      const float d6[2] = {gz[0] - hzy.x, gz[1] - hzy.y};          // dHz/dy
      const float d7[2] = {gy[0] - c_h2y[0], gy[1] - c_h2y[1]};    // dHy/dz
      const float d8[2] = {gx[0] - c_h2x[0], gx[1] - c_h2x[1]};    // dHx/dz
      const float d9[2] = {gz[0] - hzx, gz[1] - gz[0]};            // dHz/dx
      const float d10[2] = {gy[0] - hyx, gy[1] - gy[0]};           // dHy/dx
      const float d11[2] = {gx[0] - hxy.x, gx[1] - hxy.y};         // dHx/dy
      float ex[2], ey[2], ez[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float c0 = d6[c] - d7[c], c1 = d8[c] - d9[c], c2 = d10[c] - d11[c];
        ex[c] = __fadd_rn(c_e1x[c], inc_of<EX>(__fmul_rn(c_cb2[c], c0), a));
        ey[c] = __fadd_rn(c_e1y[c], inc_of<EX>(__fmul_rn(c_cb2[c], c1), a));
        ez[c] = __fadd_rn(c_e1z[c], inc_of<EX>(__fmul_rn(c_cb2[c], c2), a));
      }
      const long long q = (long long)(p - 2) * g.plane + qxy;
      ST2(Fn, q, ex[0], ex[1], true, true);
      ST2(Fn + nc, q, ey[0], ey[1], true, true);
      ST2(Fn + 2 * nc, q, ez[0], ez[1], true, true);
    }
    // ---- carry the levels one plane on ----
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      c_h2x[c] = gx[c]; c_h2y[c] = gy[c];
      c_e1x[c] = ux[c]; c_e1y[c] = uy[c]; c_e1z[c] = uz[c];
      c_h1x[c] = fx[c]; c_h1y[c] = fy[c]; c_h1z[c] = fz[c];
      c_cb2[c] = c_cb1[c]; c_cb1[c] = n_cb[c];
    }
    if (++stg == S) { stg = 0; par ^= 1u; }
  }
}

template <class KT, class... Args>
static cudaError_t launch_f2(KT kernel, dim3 grid, dim3 block, int smem, cudaStream_t s,
                             Args... args) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e) return e;
  kernel<<<grid, block, smem, s>>>(args...);
  return cudaGetLastError();
}

}  // namespace fwd2s

using namespace fwd2s;

RevUnits deep_units(const Geo& g, int zcs) {
  RevUnits U = rev_units(g, zcs);
  const int P = g.P, zc = zcs > 0 ? zcs : g.nz;
  auto up = [](int need, int t) { return (need + t - 1) / t; };   // first tile with t0 >= need
  // x: R3 spans [x0 - 2, x0 + 34); y: [y0 - 2, y0 + 9); z: planes k0 - 2 .. k1
  U.ix0 = up(P + 2, TW);
  U.ix1 = g.nx - P - 34 >= 0 ? (g.nx - P - 34) / TW + 1 : 0;
  U.iy0 = up(P + 2, TY);
  U.iy1 = g.ny - P - 9 >= 0 ? (g.ny - P - 9) / TY + 1 : 0;
  U.iz0 = up(P + 2, zc);
  U.iz1 = (g.nz - P - 1) / zc;   // full chunks ending at or below nz - P - 1
  if (U.ix1 <= U.ix0 || U.iy1 <= U.iy0 || U.iz1 <= U.iz0 || g.nx - 2 * P <= 0 ||
      g.ny - 2 * P <= 0 || g.nz - 2 * P <= 0)
    U.ix0 = U.ix1 = U.iy0 = U.iy1 = U.iz0 = U.iz1 = 0;
  return U;
}

cudaError_t launch_fwd_2step(const Fwd2Maps& m, const StepArgs& a, const RevUnits& U,
                             cudaStream_t s) {
  constexpr int S = 3;
  if (!a.Fn || !a.Fm || a.zcs <= 0 || a.zchunk <= 0) return cudaErrorInvalidValue;
  if (U.ix1 <= U.ix0 || U.iy1 <= U.iy0 || U.iz1 <= U.iz0) return cudaSuccess;
  const int Z0 = U.iz0 * a.zcs, Z1 = U.iz1 * a.zcs < a.g.nz ? U.iz1 * a.zcs : a.g.nz;
  const dim3 grid(U.ix1 - U.ix0, U.iy1 - U.iy0, (Z1 - Z0 + a.zchunk - 1) / a.zchunk);
  StepArgs b = a;
  b.U = U;
  const dim3 block(THREADS);
  if (a.xq)
    return launch_f2(k_fwd_2step<S, true>, grid, block, L2S<S>::smem(), s, m, b);
  return launch_f2(k_fwd_2step<S, false>, grid, block, L2S<S>::smem(), s, m, b);
}

}  // namespace fdtd
