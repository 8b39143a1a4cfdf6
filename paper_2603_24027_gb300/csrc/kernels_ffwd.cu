// kernels_ffwd.cu -- one launch per forward time step, two x-cells per thread.
//
// The forward H and E half-steps of one time step fused into a single pass
// over the grid: (E^n, Ht^{n-1/2}, psi) in the input buffers ->
// (E^{n+1}, Ht^{n+1/2}, psi) in the output buffers, so the state is read once
// and written once per step (52 B per cell plus the CPML auxiliaries) instead
// of twice (76 B) with two launches.
//
// A CTA owns a 32 x TY tile and a z chunk.  The E update of a cell needs
// Ht^{n+1/2} at its -x and -y neighbours, so the CTA computes Ht^{n+1/2} on
// the tile plus a one-cell halo (cells x0-2 .. x0+31, y0-1 .. y0+TY-1: pairs
// of x-cells stay 8-byte aligned) and keeps it in a shared-memory tile; halo
// values are recomputed from the same inputs as their owner CTA computes them
// (bit-identical), only owners write them.  Along z the update of plane k
// needs Ht(k) and Ht(k-1): one plane per iteration as in kernels_lag2.cu,
// iteration p finishes Ht(p-1) with E(p), then updates E(p-1), then starts
// Ht(p); the chunk's first plane k0-1 is computed but not written.  Every
// stage holds plane p's wide E box, Ht box and psi_H boxes, and plane p-1's
// own E, cb and psi_E boxes (read again from L2 rather than kept in
// registers).  The per-cell arithmetic is the sequence of rounded operations
// of every other variant, so the fields are bit-identical.
#include <cudaTypedefs.h>

#include "lag_common.cuh"

namespace fdtd {

namespace ffwd {

__device__ __forceinline__ float2 ld2(const float* b, int i) {
  return *reinterpret_cast<const float2*>(b + i);
}
__device__ __forceinline__ void st2(float* p, long long q, float u, float v, bool f0, bool f1) {
  if (f0 && f1) {
    *reinterpret_cast<float2*>(p + q) = make_float2(u, v);
  } else {
    if (f0) p[q] = u;
    if (f1) p[q + 1] = v;
  }
}
__device__ __forceinline__ float cpml(float d, float psi_old, float b, float a, float kv, float* s) {
  const float t = __fmaf_rn(b, psi_old, __fmul_rn(a, d));
  *s = t;
  return __fmaf_rn(kv, d, t);
}

// Stage layout (byte offsets) and thread counts for a 32 x TY tile.
template <int TY, int S>
struct L {
  static constexpr int EW = 40, ER = TY + 2;   // E box: x0-4 .. x0+35, y0-1 .. y0+TY
  static constexpr int HW = 36, HR = TY + 1;   // Ht / psi_H box: x0-4 .. x0+31, y0-1 .. y0+TY-1
  static constexpr int EP = EW * ER, HP = HW * HR, OP = 32 * TY;
  static constexpr int E = 0;
  static constexpr int H = E + r128(3 * EP * 4);
  static constexpr int PHX = H + r128(3 * HP * 4);
  static constexpr int PHY = PHX + r128(2 * HP * 4);
  static constexpr int PHZ = PHY + r128(2 * HP * 4);
  static constexpr int EO = PHZ + r128(2 * HP * 4);     // plane p-1
  static constexpr int CB = EO + r128(3 * OP * 4);
  static constexpr int PEX = CB + r128(OP * 4);
  static constexpr int PEY = PEX + r128(2 * OP * 4);
  static constexpr int PEZ = PEY + r128(2 * OP * 4);
  static constexpr int STAGE = PEZ + r128(2 * OP * 4);
  static constexpr int TW_ = 34, TR = TY + 1;           // Ht^{n+1/2} tile: x0-2 .., y0-1 ..
  static constexpr int TP = TW_ * TR;
  static constexpr int TILES = S * STAGE;               // two tiles x 3 components
  static constexpr int BARS = TILES + r128(2 * 3 * TP * 4);
  static constexpr int RED = BARS + 64;
  static int smem() { return RED + 64; }
  static constexpr int NH = 17 * TR;                    // Ht pairs of the tile + halo
  static constexpr int NE = 16 * TY;                    // E pairs of the tile
  static constexpr int NT = (NH + 31) / 32 * 32;        // threads (whole warps)
};

}  // namespace ffwd

using namespace ffwd;

template <int TY, int S>
__global__ void __launch_bounds__(ffwd::L<TY, S>::NT)
    k_ffwd(const __grid_constant__ FFMaps m, StepArgs a, float* __restrict__ Fo,
           float* __restrict__ psiO) {
  typedef ffwd::L<TY, S> Y;
  static_assert(Y::NT >= Y::NE, "every E pair has a thread");
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  const int p0_ = k0 - 1, p1_ = k1;
  // ---- this thread's Ht pair (tile + halo) and E pair (tile)
  const bool hact = tid < Y::NH;
  const int hr = tid / 17, hc = tid - hr * 17;
  const int hx = x0 - 2 + 2 * hc, hy = y0 - 1 + hr;
  const bool hyin = hact && hy >= 0 && hy < g.ny;
  const bool hv0 = hyin && hx >= 0 && hx < g.nx, hv1 = hyin && hx + 1 >= 0 && hx + 1 < g.nx;
  const bool hown0 = hv0 && hx >= x0 && hy >= y0, hown1 = hv1 && hx + 1 >= x0 && hy >= y0;
  const bool eact = tid < Y::NE;
  const int er = tid / 16, ec = tid - er * 16;
  const int ex = x0 + 2 * ec, ey = y0 + er;
  const bool ev0 = eact && ex < g.nx && ey < g.ny, ev1 = ev0 && ex + 1 < g.nx;
  // tiles touching a slab (Ht region and E tile)
  const bool htx = tile_in_slab(max(x0 - 2, 0), min(x0 + 31, g.nx - 1), g.nx, g.P);
  const bool hty = tile_in_slab(max(y0 - 1, 0), min(y0 + TY - 1, g.ny - 1), g.ny, g.P);
  const bool etx = tile_in_slab(x0, min(x0 + 31, g.nx - 1), g.nx, g.P);
  const bool ety = tile_in_slab(y0, min(y0 + TY - 1, g.ny - 1), g.ny, g.P);
  uint64_t* bars = reinterpret_cast<uint64_t*>(dsm + Y::BARS);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int p, unsigned char* st, uint64_t* bar) {
    const bool hb = p < k1;                      // Ht(p) is started
    const bool eb = p > k0;                      // E(p-1) is updated
    const bool hzs = hb && p >= 0 && p < g.nz && in_slab(p, g.nz, g.P);
    const bool ezs = eb && in_slab(p - 1, g.nz, g.P);
    uint32_t bytes = 3 * Y::EP * 4 + (hb ? 3 * Y::HP * 4 : 0) + (hb && htx ? 2 * Y::HP * 4 : 0) +
                     (hb && hty ? 2 * Y::HP * 4 : 0) + (hzs ? 2 * Y::HP * 4 : 0) +
                     (eb ? 4 * Y::OP * 4 : 0) + (eb && etx ? 2 * Y::OP * 4 : 0) +
                     (eb && ety ? 2 * Y::OP * 4 : 0) + (ezs ? 2 * Y::OP * 4 : 0);
    mbar_expect_tx(bar, bytes);
    tma_load_4d(st + Y::E, &m.Ew, bar, x0 - 4, y0 - 1, p, 0);
    if (hb) tma_load_4d(st + Y::H, &m.Hb, bar, x0 - 4, y0 - 1, p, 3);
    if (hb && htx) tma_load_4d(st + Y::PHX, &m.Ph, bar, x0 - 4, y0 - 1, p, 0);
    if (hb && hty) tma_load_4d(st + Y::PHY, &m.Ph, bar, x0 - 4, y0 - 1, p, 4);
    if (hzs) tma_load_4d(st + Y::PHZ, &m.Ph, bar, x0 - 4, y0 - 1, p, 8);
    if (eb) {
      tma_load_4d(st + Y::EO, &m.Eo, bar, x0, y0, p - 1, 0);
      tma_load_4d(st + Y::CB, &m.cbo, bar, x0, y0, p - 1, 0);
    }
    if (eb && etx) tma_load_4d(st + Y::PEX, &m.Pe, bar, x0, y0, p - 1, 2);
    if (eb && ety) tma_load_4d(st + Y::PEY, &m.Pe, bar, x0, y0, p - 1, 6);
    if (ezs) tma_load_4d(st + Y::PEZ, &m.Pe, bar, x0, y0, p - 1, 10);
  };
  if (tid == 0)
    for (int i = 0; i < S && p0_ + i <= p1_; ++i) issue(p0_ + i, dsm + i * Y::STAGE, bars + i);
  // ---- CPML profiles: H side for the Ht pair, E side for the E pair
  const bool hsx0 = hv0 && in_slab(hx, g.nx, g.P), hsx1 = hv1 && in_slab(hx + 1, g.nx, g.P);
  const bool hsy = hyin && in_slab(hy, g.ny, g.P);
  float hbx0 = 0.f, hax0 = 0.f, hkx0 = 1.f, hbx1 = 0.f, hax1 = 0.f, hkx1 = 1.f;
  float hby = 0.f, hay = 0.f, hky = 1.f;
  if (hsx0) { hbx0 = prof(g, 0, PR_BH, hx); hax0 = prof(g, 0, PR_AH, hx); hkx0 = prof(g, 0, PR_KH, hx); }
  if (hsx1) { hbx1 = prof(g, 0, PR_BH, hx + 1); hax1 = prof(g, 0, PR_AH, hx + 1); hkx1 = prof(g, 0, PR_KH, hx + 1); }
  if (hsy) { hby = prof(g, 1, PR_BH, hy); hay = prof(g, 1, PR_AH, hy); hky = prof(g, 1, PR_KH, hy); }
  const bool esx0 = ev0 && in_slab(ex, g.nx, g.P), esx1 = ev1 && in_slab(ex + 1, g.nx, g.P);
  const bool esy = ev0 && in_slab(ey, g.ny, g.P);
  float ebx0 = 0.f, eax0 = 0.f, ekx0 = 1.f, ebx1 = 0.f, eax1 = 0.f, ekx1 = 1.f;
  float eby = 0.f, eay = 0.f, eky = 1.f;
  if (esx0) { ebx0 = prof(g, 0, PR_BE, ex); eax0 = prof(g, 0, PR_AE, ex); ekx0 = prof(g, 0, PR_KE, ex); }
  if (esx1) { ebx1 = prof(g, 0, PR_BE, ex + 1); eax1 = prof(g, 0, PR_AE, ex + 1); ekx1 = prof(g, 0, PR_KE, ex + 1); }
  if (esy) { eby = prof(g, 1, PR_BE, ey); eay = prof(g, 1, PR_AE, ey); eky = prof(g, 1, PR_KE, ey); }
  const int eb_ = hr * Y::EW + 2 * hc + 2;     // Ht pair in the E box
  const int hb_ = hr * Y::HW + 2 * hc + 2;     // Ht pair in the Ht / psi_H boxes
  const int tb_ = hr * Y::TW_ + 2 * hc;        // Ht pair in the Ht^{n+1/2} tile
  const int te_ = (er + 1) * Y::TW_ + 2 * ec + 2;   // E pair in the Ht^{n+1/2} tile
  const int ob_ = er * 32 + 2 * ec;            // E pair in own boxes
  const long long nc = g.nc;
  float* const Hx = Fo + 3 * nc;
  float* const Hy = Hx + nc;
  float* const Hz = Hy + nc;
  float* const Ex = Fo;
  float* const Ey = Ex + nc;
  float* const Ez = Ey + nc;
  const long long hq = (long long)hy * g.px + hx;   // Ht pair within a plane
  const long long eq = (long long)ey * g.px + ex;   // E pair within a plane
  float* tiles = reinterpret_cast<float*>(dsm + Y::TILES);
  double* red = reinterpret_cast<double*>(dsm + Y::RED);
  // carried partial Ht(p-1) of the Ht pair
  float c_ex[2] = {0.f, 0.f}, c_ey[2] = {0.f, 0.f}, c_t0[2] = {0.f, 0.f}, c_t3[2] = {0.f, 0.f};
  float c_t4[2] = {0.f, 0.f}, c_t5[2] = {0.f, 0.f}, c_hx[2] = {0.f, 0.f}, c_hy[2] = {0.f, 0.f};
  float c_hz[2] = {0.f, 0.f}, c_pz0[2] = {0.f, 0.f}, c_pz1[2] = {0.f, 0.f};
  double lsum = 0.0;
  int stg = 0;
  uint32_t par = 0;
  bool ok = true;
  for (int p = p0_; p <= p1_; ++p) {
    unsigned char* st = dsm + stg * Y::STAGE;
    if (!mbar_wait(bars + stg, par, kWaitCycles)) ok = false;
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        atomicOr(a.err, ERR_TIMEOUT);
        for (int i = 0; i < S && p + i <= p1_; ++i) {
          int s = stg + i;
          uint32_t ph = par;
          if (s >= S) { s -= S; ph ^= 1u; }
          mbar_wait(&bars[s], ph, kWaitCycles);
        }
      }
      return;
    }
    const float* Eb = reinterpret_cast<const float*>(st + Y::E);
    // ---- (1) finish Ht(p-1) with dEy/dz, dEx/dz; keep it in tile (p-1) & 1
    if (p > p0_ && hact) {
      const int k = p - 1;
      const float2 ex2 = ld2(Eb, eb_), ey2 = ld2(Eb + Y::EP, eb_);
      float t1[2] = {ey2.x - c_ey[0], ey2.y - c_ey[1]};
      float t2[2] = {ex2.x - c_ex[0], ex2.y - c_ex[1]};
      const bool wr = k >= k0;   // the chunk's first plane k0-1 belongs to the chunk below
      if (k >= 0 && in_slab(k, g.nz, g.P)) {
        const float bz = prof(g, 2, PR_BH, k), az = prof(g, 2, PR_AH, k), kz = prof(g, 2, PR_KH, k);
        float s1[2], s2[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          t1[c] = cpml(t1[c], c_pz0[c], bz, az, kz, &s1[c]);
          t2[c] = cpml(t2[c], c_pz1[c], bz, az, kz, &s2[c]);
        }
        if (wr) {
          const long long q = (long long)k * g.plane + hq;
          st2(psiO + 8 * nc, q, s1[0], s1[1], hown0, hown1);
          st2(psiO + 9 * nc, q, s2[0], s2[1], hown0, hown1);
        }
      }
      float nx_[2], ny_[2], nz_[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float cx = c_t0[c] - t1[c], cy = t2[c] - c_t3[c], cz = c_t4[c] - c_t5[c];
        nx_[c] = __fsub_rn(c_hx[c], __fmul_rn(g.S, cx));
        ny_[c] = __fsub_rn(c_hy[c], __fmul_rn(g.S, cy));
        nz_[c] = __fsub_rn(c_hz[c], __fmul_rn(g.S, cz));
      }
      // cells outside the grid (the plane below z = 0 included) hold zero: the
      // E update reads them as the zero-padding neighbours of the first
      // row / column / plane
      float* T = tiles + (k & 1) * 3 * Y::TP;
      const bool in0 = hv0 && k >= 0, in1 = hv1 && k >= 0;
      *reinterpret_cast<float2*>(T + tb_) = make_float2(in0 ? nx_[0] : 0.f, in1 ? nx_[1] : 0.f);
      *reinterpret_cast<float2*>(T + Y::TP + tb_) =
          make_float2(in0 ? ny_[0] : 0.f, in1 ? ny_[1] : 0.f);
      *reinterpret_cast<float2*>(T + 2 * Y::TP + tb_) =
          make_float2(in0 ? nz_[0] : 0.f, in1 ? nz_[1] : 0.f);
      if (wr && (hown0 || hown1)) {
        const long long q = (long long)k * g.plane + hq;
        st2(Hx, q, nx_[0], nx_[1], hown0, hown1);
        st2(Hy, q, ny_[0], ny_[1], hown0, hown1);
        st2(Hz, q, nz_[0], nz_[1], hown0, hown1);
      }
    }
    __syncthreads();
    // ---- (2) E(p-1) from Ht^{n+1/2}(p-1), Ht^{n+1/2}(p-2) in the tiles
    if (p > k0 && ev0) {
      const int k = p - 1;
      const float* T = tiles + (k & 1) * 3 * Y::TP;         // Ht(k)
      const float* Tm = tiles + ((k + 1) & 1) * 3 * Y::TP;  // Ht(k-1)
      const float2 hx2 = ld2(T, te_), hy2 = ld2(T + Y::TP, te_), hz2 = ld2(T + 2 * Y::TP, te_);
      const float hx[2] = {hx2.x, hx2.y}, hy[2] = {hy2.x, hy2.y}, hz[2] = {hz2.x, hz2.y};
      const float2 hzy = ld2(T + 2 * Y::TP, te_ - Y::TW_), hxy = ld2(T, te_ - Y::TW_);
      const float hzx = T[2 * Y::TP + te_ - 1], hyx = T[Y::TP + te_ - 1];
      const float2 pxm = ld2(Tm, te_), pym = ld2(Tm + Y::TP, te_);
      const float d6[2] = {hz[0] - hzy.x, hz[1] - hzy.y};   // dHz/dy
      const float d7[2] = {hy[0] - pym.x, hy[1] - pym.y};   // dHy/dz
      const float d8[2] = {hx[0] - pxm.x, hx[1] - pxm.y};   // dHx/dz
      const float d9[2] = {hz[0] - hzx, hz[1] - hz[0]};     // dHz/dx
      const float d10[2] = {hy[0] - hyx, hy[1] - hy[0]};    // dHy/dx
      const float d11[2] = {hx[0] - hxy.x, hx[1] - hxy.y};  // dHx/dy
      const bool sz = in_slab(k, g.nz, g.P);
      const long long q = (long long)k * g.plane + eq;
      float c0[2], c1[2], c2[2];
      if (!(esx0 || esx1 || esy || sz)) {
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
        if (esx0 || esx1) {
          const float* P = reinterpret_cast<const float*>(st + Y::PEX);
          const float2 p0 = ld2(P, ob_), p1 = ld2(P + Y::OP, ob_);
          float s9[2] = {0.f, 0.f}, s10[2] = {0.f, 0.f};
          if (esx0) {
            t9[0] = cpml(d9[0], p0.x, ebx0, eax0, ekx0, &s9[0]);
            t10[0] = cpml(d10[0], p1.x, ebx0, eax0, ekx0, &s10[0]);
          }
          if (esx1) {
            t9[1] = cpml(d9[1], p0.y, ebx1, eax1, ekx1, &s9[1]);
            t10[1] = cpml(d10[1], p1.y, ebx1, eax1, ekx1, &s10[1]);
          }
          st2(psiO + 2 * nc, q, s9[0], s9[1], esx0, esx1);
          st2(psiO + 3 * nc, q, s10[0], s10[1], esx0, esx1);
        }
        if (esy) {
          const float* P = reinterpret_cast<const float*>(st + Y::PEY);
          const float2 p0 = ld2(P, ob_), p1 = ld2(P + Y::OP, ob_);
          const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
          float s6[2], s11[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            t6[c] = cpml(d6[c], q0[c], eby, eay, eky, &s6[c]);
            t11[c] = cpml(d11[c], q1[c], eby, eay, eky, &s11[c]);
          }
          st2(psiO + 6 * nc, q, s6[0], s6[1], true, ev1);
          st2(psiO + 7 * nc, q, s11[0], s11[1], true, ev1);
        }
        if (sz) {
          const float* P = reinterpret_cast<const float*>(st + Y::PEZ);
          const float bz = prof(g, 2, PR_BE, k), az = prof(g, 2, PR_AE, k), kz = prof(g, 2, PR_KE, k);
          const float2 p0 = ld2(P, ob_), p1 = ld2(P + Y::OP, ob_);
          const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
          float s7[2], s8[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            t7[c] = cpml(d7[c], q0[c], bz, az, kz, &s7[c]);
            t8[c] = cpml(d8[c], q1[c], bz, az, kz, &s8[c]);
          }
          st2(psiO + 10 * nc, q, s7[0], s7[1], true, ev1);
          st2(psiO + 11 * nc, q, s8[0], s8[1], true, ev1);
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
          const float w = (c == 0 || ev1) ? src_wt(a.src, ex + c, ey, k) : 0.f;
          if (w != 0.f) {
            const float wj = __fmul_rn(w, a.jn);
            if (a.src.comp == 0) c0[c] = __fsub_rn(c0[c], wj);
            else if (a.src.comp == 1) c1[c] = __fsub_rn(c1[c], wj);
            else c2[c] = __fsub_rn(c2[c], wj);
          }
        }
      }
      const float* Eo = reinterpret_cast<const float*>(st + Y::EO);
      const float2 cb2 = ld2(reinterpret_cast<const float*>(st + Y::CB), ob_);
      const float2 e0 = ld2(Eo, ob_), e1 = ld2(Eo + Y::OP, ob_), e2 = ld2(Eo + 2 * Y::OP, ob_);
      const float cbv[2] = {cb2.x, cb2.y};
      const float eo0[2] = {e0.x, e0.y}, eo1[2] = {e1.x, e1.y}, eo2[2] = {e2.x, e2.y};
      float nex[2], ney[2], nez[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        nex[c] = __fadd_rn(eo0[c], __fmul_rn(cbv[c], c0[c]));
        ney[c] = __fadd_rn(eo1[c], __fmul_rn(cbv[c], c1[c]));
        nez[c] = __fadd_rn(eo2[c], __fmul_rn(cbv[c], c2[c]));
      }
      st2(Ex, q, nex[0], nex[1], true, ev1);
      st2(Ey, q, ney[0], ney[1], true, ev1);
      st2(Ez, q, nez[0], nez[1], true, ev1);
      if (a.det.kind) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          int u, v;
          if ((c == 0 || ev1) && on_plane(a.det.axis, a.det.index, a.det.u0, a.det.u1, a.det.v0,
                                          a.det.v1, ex + c, ey, k, &u, &v)) {
            if (a.det.kind == 1) {
              lsum += (double)nex[c] * nex[c] + (double)ney[c] * ney[c] + (double)nez[c] * nez[c];
            } else {
              const int ax_ = a.det.axis;
              const float Eb_ = ax_ == 0 ? ney[c] : (ax_ == 1 ? nez[c] : nex[c]);
              const float Ec2 = ax_ == 0 ? nez[c] : (ax_ == 1 ? nex[c] : ney[c]);
              const float Hb2 = ax_ == 0 ? hy[c] : (ax_ == 1 ? hz[c] : hx[c]);
              const float Hc2 = ax_ == 0 ? hz[c] : (ax_ == 1 ? hx[c] : hy[c]);
              lsum += (double)Eb_ * Hc2 - (double)Ec2 * Hb2;
            }
          }
        }
      }
    }
    // ---- (3) start Ht(p): x and y derivatives of E(p), their psi updates
    if (p < k1 && hact) {
      const float2 ex2 = ld2(Eb, eb_), ey2 = ld2(Eb + Y::EP, eb_), ez2 = ld2(Eb + 2 * Y::EP, eb_);
      const float2 ezy = ld2(Eb + 2 * Y::EP, eb_ + Y::EW), exy = ld2(Eb, eb_ + Y::EW);
      const float ezx = Eb[2 * Y::EP + eb_ + 2], eyx = Eb[Y::EP + eb_ + 2];
      float t0[2] = {ezy.x - ez2.x, ezy.y - ez2.y};     // dEz/dy
      float t3[2] = {ez2.y - ez2.x, ezx - ez2.y};       // dEz/dx
      float t4[2] = {ey2.y - ey2.x, eyx - ey2.y};       // dEy/dx
      float t5[2] = {exy.x - ex2.x, exy.y - ex2.y};     // dEx/dy
      const bool wr = p >= k0;
      const long long q = (long long)p * g.plane + hq;
      if (hsx0 || hsx1) {
        const float* P = reinterpret_cast<const float*>(st + Y::PHX);
        const float2 p0 = ld2(P, hb_), p1 = ld2(P + Y::HP, hb_);
        float s3[2] = {0.f, 0.f}, s4[2] = {0.f, 0.f};
        if (hsx0) {
          t3[0] = cpml(t3[0], p0.x, hbx0, hax0, hkx0, &s3[0]);
          t4[0] = cpml(t4[0], p1.x, hbx0, hax0, hkx0, &s4[0]);
        }
        if (hsx1) {
          t3[1] = cpml(t3[1], p0.y, hbx1, hax1, hkx1, &s3[1]);
          t4[1] = cpml(t4[1], p1.y, hbx1, hax1, hkx1, &s4[1]);
        }
        if (wr) {
          st2(psiO, q, s3[0], s3[1], hsx0 && hown0, hsx1 && hown1);
          st2(psiO + nc, q, s4[0], s4[1], hsx0 && hown0, hsx1 && hown1);
        }
      }
      if (hsy) {
        const float* P = reinterpret_cast<const float*>(st + Y::PHY);
        const float2 p0 = ld2(P, hb_), p1 = ld2(P + Y::HP, hb_);
        const float q0[2] = {p0.x, p0.y}, q1[2] = {p1.x, p1.y};
        float s0[2], s5[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          t0[c] = cpml(t0[c], q0[c], hby, hay, hky, &s0[c]);
          t5[c] = cpml(t5[c], q1[c], hby, hay, hky, &s5[c]);
        }
        if (wr) {
          st2(psiO + 4 * nc, q, s0[0], s0[1], hown0, hown1);
          st2(psiO + 5 * nc, q, s5[0], s5[1], hown0, hown1);
        }
      }
      const float* Hb = reinterpret_cast<const float*>(st + Y::H);
      const float2 h0 = ld2(Hb, hb_), h1 = ld2(Hb + Y::HP, hb_), h2 = ld2(Hb + 2 * Y::HP, hb_);
      c_ex[0] = ex2.x; c_ex[1] = ex2.y;
      c_ey[0] = ey2.x; c_ey[1] = ey2.y;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        c_t0[c] = t0[c];
        c_t3[c] = t3[c];
        c_t4[c] = t4[c];
        c_t5[c] = t5[c];
      }
      c_hx[0] = h0.x; c_hx[1] = h0.y;
      c_hy[0] = h1.x; c_hy[1] = h1.y;
      c_hz[0] = h2.x; c_hz[1] = h2.y;
      if (p >= 0 && in_slab(p, g.nz, g.P)) {
        const float* P = reinterpret_cast<const float*>(st + Y::PHZ);
        const float2 p0 = ld2(P, hb_), p1 = ld2(P + Y::HP, hb_);
        c_pz0[0] = p0.x; c_pz0[1] = p0.y;
        c_pz1[0] = p1.x; c_pz1[1] = p1.y;
      } else {
        c_pz0[0] = c_pz0[1] = c_pz1[0] = c_pz1[1] = 0.f;
      }
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
      for (int wv = 0; wv < Y::NT / 32; ++wv) t += red[wv];
      if (t != 0.0) atomicAdd(a.obj, t);
    }
  }
}

template <int TY, int S>
static cudaError_t launch_ffwd_t(const FFMaps& m, const StepArgs& a, float* Fo, float* psiO,
                                 cudaStream_t s) {
  typedef ffwd::L<TY, S> Y;
  dim3 grid((a.g.nx + 31) / 32, (a.g.ny + TY - 1) / TY, (a.g.nz + a.zchunk - 1) / a.zchunk);
  const int sm = Y::smem();
  cudaError_t e = cudaFuncSetAttribute(k_ffwd<TY, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e) return e;
  k_ffwd<TY, S><<<grid, Y::NT, sm, s>>>(m, a, Fo, psiO);
  return cudaGetLastError();
}

// Tile heights 4 and 8 (others run with 8), 2 or 3 stages.
cudaError_t launch_ffwd(const FFMaps& m, const StepArgs& a, float* Fo, float* psiO,
                        cudaStream_t s) {
  if (a.tile_y <= 4)
    return a.stages >= 3 ? launch_ffwd_t<4, 3>(m, a, Fo, psiO, s) : launch_ffwd_t<4, 2>(m, a, Fo, psiO, s);
  return a.stages >= 3 ? launch_ffwd_t<8, 3>(m, a, Fo, psiO, s) : launch_ffwd_t<8, 2>(m, a, Fo, psiO, s);
}

// ---------------------------------------------------------- tensor maps ---
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn_ff() {
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

static cudaError_t enc_ff(CUtensorMap* m, const float* base, const Geo& g, int ncomp, int bx,
                          int by, int bc) {
  auto fn = encode_fn_ff();
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

cudaError_t encode_ffwd_maps(const float* F, const float* cb, const float* psiA, const Geo& g,
                             int ty, FFMaps* m) {
  const int TY = ty <= 4 ? 4 : 8;
  cudaError_t e;
  if ((e = enc_ff(&m->Ew, F, g, 6, 40, TY + 2, 3))) return e;
  if ((e = enc_ff(&m->Hb, F, g, 6, 36, TY + 1, 3))) return e;
  if ((e = enc_ff(&m->Eo, F, g, 6, 32, TY, 3))) return e;
  if ((e = enc_ff(&m->cbo, cb, g, 1, 32, TY, 1))) return e;
  if ((e = enc_ff(&m->Ph, psiA, g, 12, 36, TY + 1, 2))) return e;
  return enc_ff(&m->Pe, psiA, g, 12, 32, TY, 2);
}

}  // namespace fdtd
