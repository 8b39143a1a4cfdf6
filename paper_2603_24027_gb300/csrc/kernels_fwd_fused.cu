// kernels_fwd_fused.cu -- one forward time step of the CPML-free units in one launch.
//
// A forward step n of the leapfrog (the simulation whose gradient Sec. 2
// computes):
//     Ht^{n+1/2} = Ht^{n-1/2} - S curl E^n              (forward differences)
//     E^{n+1}    = E^n + cb (curl Ht^{n+1/2} - J)       (backward differences)
// The split half-steps (kernels_lag2.cu) read E and Ht in both launches, 76 B
// per interior cell.  Here a CTA runs both half-steps of its unit in one
// pass: it reads E^n, Ht^{n-1/2} and cb once and writes E^{n+1} and
// Ht^{n+1/2} once (52 B) into the other buffer of a ping-pong pair, so no
// CTA reads a value another CTA of the launch has already replaced.
//
// E^{n+1} of a cell needs Ht^{n+1/2} at -x, -y and -z.  Across z it comes one
// iteration later (the E update lags one plane); across x and y the CTA
// computes Ht^{n+1/2} itself on a one-cell halo of its tile (a fifth warp: a
// row of 16 pairs at y0-1 and a column of 8 cells at x0-1), from the same
// staged inputs.  Every cell sees the same sequence of explicitly rounded
// operations as in the split kernels, so the fields are bit-identical to
// theirs.
//
// The launch covers the units without a CPML term ([ix0, ix1) x [iy0, iy1) x
// [iz0, iz1) of RevUnits): every cell and neighbour a CTA touches is in the
// interior and inside the grid, so no boundary case arises.  The host gives
// it only grids whose source and detector lie outside those units; the
// split kernels run the other units (z-only and ring) from and into the same
// buffer pair.
#include <cudaTypedefs.h>

#include "lag_common.cuh"

namespace fdtd {

using namespace lag2;

namespace fwdf {

// Shared memory (byte offsets): S stages of an E box (TW+8) x (TY+2) at
// (x0-4, y0-1), an Ht box (TW+4) x (TY+1) at (x0-4, y0-1) (3 components
// each) and a cb box TW x TY at (x0, y0); the stages' mbarriers right after
// them (where ring_init puts them); then Ht^{n+1/2} of one plane on the tile
// and its -x / -y halo, [3][TY+1][TW+4] at (x0-4, y0-1).
template <int TY, int S, int TW>
struct FL {
  static constexpr int WW = TW + 8, WR = TY + 2, WP = WW * WR;
  static constexpr int HW = TW + 4, HR = TY + 1, HP = HW * HR;
  static constexpr int OP = TW * TY;
  static constexpr int E = 0;
  static constexpr int H = E + r128(3 * WP * 4);
  static constexpr int CB = H + r128(3 * HP * 4);
  static constexpr int STAGE = CB + r128(OP * 4);
  static constexpr int BARS = S * STAGE;
  static constexpr int SH = r128(BARS + 8 * S);
  static int smem() { return SH + 3 * HP * 4; }
};

static_assert(FL<8, 3, 32>::SH >= FL<8, 3, 32>::BARS + 8 * 3, "SH after the barriers");

template <int TY, int S, int TW, bool EX>
__global__ void __launch_bounds__(TW / 2 * (TY + 2), 6)
k_fwd_fused(const __grid_constant__ RevMaps m, StepArgs a) {
  typedef FL<TY, S, TW> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * (TW / 2) + tx;
  const int x0 = (blockIdx.x + a.t0x) * TW, y0 = (blockIdx.y + a.t0y) * TY;
  const int k0 = (blockIdx.z + a.zc0) * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  // task: the tile's pair (main), a pair of the -y halo row, or the -x halo
  // column (pair x0-2, x0-1)
  const bool mainT = ty < TY;
  const bool rowT = ty == TY;
  const bool colT = ty == TY + 1 && tx < TY;
  const bool task = mainT || rowT || colT;
  const int x = colT ? x0 - 2 : x0 + 2 * tx;
  const int y = mainT ? y0 + ty : (rowT ? y0 - 1 : y0 + tx);
  // plane k0-1 starts Ht'(k0-1); plane p in [k0, k1) finishes Ht'(p-1),
  // updates E(p-1) (from k0+1 on) and starts Ht'(p); plane k1 finishes
  // Ht'(k1-1) and updates E(k1-1)
  const int p0_ = k0 - 1, p1_ = k1;
  uint64_t* bars = ring_init<S>(dsm, Y::STAGE);   // at Y::BARS
  auto boxes = [&](int p, auto&& f) {
    f(Y::E, &m.F40, x0 - 4, y0 - 1, p, 0, 3 * Y::WP * 4);
    if (p < k1) {
      f(Y::H, &m.F36, x0 - 4, y0 - 1, p, 3, 3 * Y::HP * 4);
      if (p >= k0) f(Y::CB, &m.cb32, x0, y0, p, 0, Y::OP * 4);
    }
  };
  auto issue = [&](int p, unsigned char* st, uint64_t* bar) {
    stage_plane(boxes, p, st, bar, false);
  };
  if (tid == 0)
    for (int i = 0; i < S && p0_ + i <= p1_; ++i) issue(p0_ + i, dsm + i * Y::STAGE, bars + i);
  const int wb = (y - y0 + 1) * Y::WW + (x - x0 + 4);   // the pair in the E box
  const int hb = (y - y0 + 1) * Y::HW + (x - x0 + 4);   // the pair in the Ht box and SH
  const int ob = (y - y0) * TW + (x - x0);               // the pair in the cb box (main)
  float* SH = reinterpret_cast<float*>(dsm + Y::SH);
  const float S_ = g.S;
  const long long nc = g.nc;
  float* const Fn = a.Fn;
  const long long qxy = (long long)y * g.px + x;
  // Ht'(p-1) in progress at the pair: E(p-1) x / y, the x / y difference
  // terms, Ht(p-1)
  float c_ex[2] = {0.f, 0.f}, c_ey[2] = {0.f, 0.f}, c_t0[2] = {0.f, 0.f}, c_t3[2] = {0.f, 0.f};
  float c_t4[2] = {0.f, 0.f}, c_t5[2] = {0.f, 0.f}, c_hx[2] = {0.f, 0.f}, c_hy[2] = {0.f, 0.f};
  float c_hz[2] = {0.f, 0.f};
  // E'(p-1) at the pair: Ez(p-1), cb(p-1) and Ht'x, Ht'y of plane p-2
  float c_ez[2] = {0.f, 0.f}, c_cb[2] = {0.f, 0.f}, c_fx[2] = {0.f, 0.f}, c_fy[2] = {0.f, 0.f};
  int stg = 0;
  uint32_t par = 0;
  bool ok = true;
  for (int p = p0_; p <= p1_; ++p) {
    unsigned char* st = dsm + stg * Y::STAGE;
    if (!mbar_wait(bars + stg, par, kWaitCycles)) ok = false;
    if (!__syncthreads_and(ok)) { ring_abort<S>(bars, stg, par, p, p1_, a.err); return; }
    const float* Eb = reinterpret_cast<const float*>(st + Y::E);
    const bool head = p < k0, tail = p == k1;
    float fx[2] = {0.f, 0.f}, fy[2] = {0.f, 0.f}, fz[2] = {0.f, 0.f};   // Ht'(p-1) at the pair
    // ---- finish Ht'(p-1) with dEy/dz and dEx/dz ----
    if (task && !head) {
      const float2 ex2 = ld2(Eb, wb), ey2 = ld2(Eb + Y::WP, wb);
      const float ex[2] = {ex2.x, ex2.y}, ey[2] = {ey2.x, ey2.y};
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float t1 = ey[c] - c_ey[c], t2 = ex[c] - c_ex[c];
        const float cx = c_t0[c] - t1, cy = t2 - c_t3[c], cz = c_t4[c] - c_t5[c];
        fx[c] = __fsub_rn(c_hx[c], inc_of<EX>(__fmul_rn(S_, cx), a));
        fy[c] = __fsub_rn(c_hy[c], inc_of<EX>(__fmul_rn(S_, cy), a));
        fz[c] = __fsub_rn(c_hz[c], inc_of<EX>(__fmul_rn(S_, cz), a));
      }
      *reinterpret_cast<float2*>(SH + hb) = make_float2(fx[0], fx[1]);
      *reinterpret_cast<float2*>(SH + Y::HP + hb) = make_float2(fy[0], fy[1]);
      *reinterpret_cast<float2*>(SH + 2 * Y::HP + hb) = make_float2(fz[0], fz[1]);
      if (mainT && p - 1 >= k0) {
        const long long qm = (long long)(p - 1) * g.plane + qxy;
        ST2(Fn + 3 * nc, qm, fx[0], fx[1], true, true);
        ST2(Fn + 4 * nc, qm, fy[0], fy[1], true, true);
        ST2(Fn + 5 * nc, qm, fz[0], fz[1], true, true);
      }
    }
    __syncthreads();   // Ht'(p-1) of the tile and its halo is in SH
    // ---- E'(p-1), one plane behind ----
    if (mainT && p - 1 >= k0) {
      const float2 hzy = ld2(SH + 2 * Y::HP, hb - Y::HW), hxy = ld2(SH, hb - Y::HW);   // -y
      const float hzx = SH[2 * Y::HP + hb - 1], hyx = SH[Y::HP + hb - 1];               // -x of cell 0
      const float d6[2] = {fz[0] - hzy.x, fz[1] - hzy.y};        // dHz/dy
      const float d7[2] = {fy[0] - c_fy[0], fy[1] - c_fy[1]};    // dHy/dz
      const float d8[2] = {fx[0] - c_fx[0], fx[1] - c_fx[1]};    // dHx/dz
      const float d9[2] = {fz[0] - hzx, fz[1] - fz[0]};          // dHz/dx
      const float d10[2] = {fy[0] - hyx, fy[1] - fy[0]};         // dHy/dx
      const float d11[2] = {fx[0] - hxy.x, fx[1] - hxy.y};       // dHx/dy
      float ex[2], ey[2], ez[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float c0 = d6[c] - d7[c], c1 = d8[c] - d9[c], c2 = d10[c] - d11[c];
        ex[c] = __fadd_rn(c_ex[c], inc_of<EX>(__fmul_rn(c_cb[c], c0), a));
        ey[c] = __fadd_rn(c_ey[c], inc_of<EX>(__fmul_rn(c_cb[c], c1), a));
        ez[c] = __fadd_rn(c_ez[c], inc_of<EX>(__fmul_rn(c_cb[c], c2), a));
      }
      const long long qm = (long long)(p - 1) * g.plane + qxy;
      ST2(Fn, qm, ex[0], ex[1], true, true);
      ST2(Fn + nc, qm, ey[0], ey[1], true, true);
      ST2(Fn + 2 * nc, qm, ez[0], ez[1], true, true);
    }
    if (mainT && !head) {   // Ht'(p-1) at the pair: the -z neighbour of E'(p)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        c_fx[c] = fx[c];
        c_fy[c] = fy[c];
      }
    }
    // ---- start Ht'(p): its x and y differences ----
    if (task && !tail) {
      const float2 ex2 = ld2(Eb, wb), ey2 = ld2(Eb + Y::WP, wb), ez2 = ld2(Eb + 2 * Y::WP, wb);
      const float2 ezy = ld2(Eb + 2 * Y::WP, wb + Y::WW), exy = ld2(Eb, wb + Y::WW);   // +y
      const float ezx = Eb[2 * Y::WP + wb + 2], eyx = Eb[Y::WP + wb + 2];               // +x of cell 1
      const float* Hb = reinterpret_cast<const float*>(st + Y::H);
      const float2 h0 = ld2(Hb, hb), h1 = ld2(Hb + Y::HP, hb), h2 = ld2(Hb + 2 * Y::HP, hb);
      c_t0[0] = ezy.x - ez2.x; c_t0[1] = ezy.y - ez2.y;   // dEz/dy
      c_t3[0] = ez2.y - ez2.x; c_t3[1] = ezx - ez2.y;     // dEz/dx
      c_t4[0] = ey2.y - ey2.x; c_t4[1] = eyx - ey2.y;     // dEy/dx
      c_t5[0] = exy.x - ex2.x; c_t5[1] = exy.y - ex2.y;   // dEx/dy
      c_ex[0] = ex2.x; c_ex[1] = ex2.y;
      c_ey[0] = ey2.x; c_ey[1] = ey2.y;
      c_hx[0] = h0.x; c_hx[1] = h0.y;
      c_hy[0] = h1.x; c_hy[1] = h1.y;
      c_hz[0] = h2.x; c_hz[1] = h2.y;
      if (mainT && !head) {
        const float2 cb2 = ld2(reinterpret_cast<const float*>(st + Y::CB), ob);
        c_ez[0] = ez2.x; c_ez[1] = ez2.y;
        c_cb[0] = cb2.x; c_cb[1] = cb2.y;
      }
    }
    __syncthreads();   // SH and the stage are free again
    if (tid == 0 && p + S <= p1_) issue(p + S, st, bars + stg);
    if (++stg == S) { stg = 0; par ^= 1u; }
  }
}

template <class KT, class... Args>
static cudaError_t launch_ff(KT kernel, dim3 grid, dim3 block, int smem, cudaStream_t s,
                             Args... args) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e) return e;
  kernel<<<grid, block, smem, s>>>(args...);
  return cudaGetLastError();
}

}  // namespace fwdf

using namespace fwdf;

cudaError_t launch_fwd_fused(const RevMaps& m, const StepArgs& a, const RevUnits& U,
                             cudaStream_t s) {
  constexpr int TW = 32, TY = 8, S = 3;
  if (a.tile_y != TY || a.tile_x != TW || !a.Fn) return cudaErrorInvalidValue;
  const dim3 grid(U.ix1 - U.ix0, U.iy1 - U.iy0, U.iz1 - U.iz0);
  if (U.ix1 <= U.ix0 || U.iy1 <= U.iy0 || U.iz1 <= U.iz0) return cudaSuccess;
  StepArgs b = a;
  b.t0x = U.ix0;
  b.t0y = U.iy0;
  b.zc0 = U.iz0;
  const dim3 block(TW / 2, TY + 2);
  if (a.xq)
    return launch_ff(k_fwd_fused<TY, S, TW, true>, grid, block, FL<TY, S, TW>::smem(), s, m, b);
  return launch_ff(k_fwd_fused<TY, S, TW, false>, grid, block, FL<TY, S, TW>::smem(), s, m, b);
}

}  // namespace fdtd
