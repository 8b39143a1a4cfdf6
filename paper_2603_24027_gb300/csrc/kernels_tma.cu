// kernels_tma.cu -- TMA-pipelined fused step kernels.
//
// Same per-cell arithmetic as the split and plain fused kernels (so all paths
// give bit-identical fields), but the z-planes a CTA needs are streamed into
// shared memory by the tensor-memory accelerator through an S-stage ring of
// mbarrier-tracked buffers: one elected thread keeps S planes in flight, so
// the bytes in flight per SM no longer depend on how many threads are
// resident.  Box loads start at x0-4 (the TMA needs the innermost coordinate
// on a 16-byte boundary) and read zeros outside the grid, which is the
// zero-padding boundary condition.
#include <cudaTypedefs.h>

#include "fdtd_internal.cuh"
#include "tma.cuh"

namespace fdtd {

// --------------------------------------------------------- tensor maps ---
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// 4D view (x, y, z, component) of `ncomp` consecutive component arrays.
static cudaError_t encode4(CUtensorMap* m, const float* base, const Geo& g, int ncomp, int bx,
                           int by, int bc) {
  auto fn = encode_fn();
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

cudaError_t encode_fwd_maps(const float* F, const float* cb, const Geo& g, int ty, FwdMaps* m) {
  cudaError_t e;
  if ((e = encode4(&m->E, F, g, 6, 40, ty + 2, 3))) return e;
  if ((e = encode4(&m->H, F, g, 6, 40, ty + 1, 3))) return e;
  return encode4(&m->cb, cb, g, 1, 32, ty, 1);
}

// ---------------------------------------------------------- forward ------
__device__ __forceinline__ float cpml_t(float d, const float* pin, float* pout, long long pi,
                                        const Geo& g, int ax, int pos, int side) {
  float b = prof(g, ax, side + 0, pos), a = prof(g, ax, side + 1, pos),
        kv = prof(g, ax, side + 2, pos);
  float s = __fmaf_rn(b, pin[pi], __fmul_rn(a, d));
  if (pout) pout[pi] = s;
  return __fmaf_rn(kv, d, s);
}

template <int TY>
struct FwdLayout {
  static constexpr int W = 40;                 // staged x range [x0-4, x0+36)
  static constexpr int ER = TY + 2;            // E rows [y0-1, y0+TY+1)
  static constexpr int HR = TY + 1;            // H rows [y0-1, y0+TY)
  static constexpr int E_FL = 3 * ER * W;
  static constexpr int H_FL = 3 * HR * W;
  static constexpr int CB_FL = TY * 32;
  static constexpr int r128(int b) { return (b + 127) / 128 * 128; }
  static constexpr int E_OFF = 0;
  static constexpr int H_OFF = r128(E_FL * 4);
  static constexpr int CB_OFF = H_OFF + r128(H_FL * 4);
  static constexpr int STAGE = CB_OFF + r128(CB_FL * 4);
  static constexpr uint32_t TX_BYTES = (E_FL + H_FL + CB_FL) * 4;
  static constexpr int SH_BYTES = r128(3 * HR * W * 4);
  static int bytes(int S) { return S * STAGE + SH_BYTES + 128 + 8 * S + 256; }
};

// Ht^{n+1/2} at one cell from staged planes: Ec/En = E^n planes k and k+1
// ([3][ER][W]), Hm = Ht^{n-1/2} plane k ([3][HR][W]); (xi, yi) = position in
// the staged region.
template <int TY>
__device__ __forceinline__ void h_from_stage(const Geo& g, const float* Ec, const float* En,
                                             const float* Hm, int xi, int yi, int x, int y, int k,
                                             const float* pin, float* pout, float h[3]) {
  typedef FwdLayout<TY> LY;
  constexpr int W = LY::W, EP = LY::ER * W, HP = LY::HR * W;
  const int e0 = yi * W + xi;
  const float ex = Ec[e0], ey = Ec[EP + e0], ez = Ec[2 * EP + e0];
  const float d0 = Ec[2 * EP + e0 + W] - ez;   // dEz/dy
  const float d1 = En[EP + e0] - ey;           // dEy/dz
  const float d2 = En[e0] - ex;                // dEx/dz
  const float d3 = Ec[2 * EP + e0 + 1] - ez;   // dEz/dx
  const float d4 = Ec[EP + e0 + 1] - ey;       // dEy/dx
  const float d5 = Ec[e0 + W] - ex;            // dEx/dy
  const bool sx = in_slab(x, g.nx, g.P), sy = in_slab(y, g.ny, g.P), sz = in_slab(k, g.nz, g.P);
  float cx, cy, cz;
  if (!(sx || sy || sz)) {
    cx = d0 - d1;
    cy = d2 - d3;
    cz = d4 - d5;
  } else {
    float t0 = d0, t1 = d1, t2 = d2, t3 = d3, t4 = d4, t5 = d5;
    if (sx) {
      t3 = cpml_t(d3, pin, pout, psi_x(g, 0, x, y, k), g, 0, x, PR_BH);
      t4 = cpml_t(d4, pin, pout, psi_x(g, 1, x, y, k), g, 0, x, PR_BH);
    }
    if (sy) {
      t0 = cpml_t(d0, pin, pout, psi_y(g, 0, x, y, k), g, 1, y, PR_BH);
      t5 = cpml_t(d5, pin, pout, psi_y(g, 1, x, y, k), g, 1, y, PR_BH);
    }
    if (sz) {
      t1 = cpml_t(d1, pin, pout, psi_z(g, 0, x, y, k), g, 2, k, PR_BH);
      t2 = cpml_t(d2, pin, pout, psi_z(g, 1, x, y, k), g, 2, k, PR_BH);
    }
    cx = t0 - t1;
    cy = t2 - t3;
    cz = t4 - t5;
  }
  const int h0 = yi * W + xi;
  h[0] = __fsub_rn(Hm[h0], __fmul_rn(g.S, cx));
  h[1] = __fsub_rn(Hm[HP + h0], __fmul_rn(g.S, cy));
  h[2] = __fsub_rn(Hm[2 * HP + h0], __fmul_rn(g.S, cz));
}

__device__ __forceinline__ float srcw_t(const Src& s, int i, int j, int k) {
  int u, v;
  if (s.kind == 0 || !on_plane(s.axis, s.index, s.u0, s.u1, s.v0, s.v1, i, j, k, &u, &v))
    return 0.f;
  return __ldg(s.w + (long long)(v - s.v0) * (s.u1 - s.u0) + (u - s.u0));
}

template <int TY, int S>
__global__ void __launch_bounds__(32 * TY) k_fwd_tma(const __grid_constant__ FwdMaps maps,
                                                    StepArgs a, float* __restrict__ Fo,
                                                    float* __restrict__ psiO) {
  typedef FwdLayout<TY> LY;
  constexpr int W = LY::W;
  constexpr int HP = LY::HR * W;
  constexpr int NT = 32 * TY;
  extern __shared__ __align__(128) unsigned char dsm[];
  float* sH = reinterpret_cast<float*>(dsm + S * LY::STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(dsm + S * LY::STAGE + LY::SH_BYTES);
  double* red = reinterpret_cast<double*>(dsm + S * LY::STAGE + LY::SH_BYTES + 128);

  const Geo& g = a.g;
  const float* __restrict__ psiI = a.psiA;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
  const int x = x0 + tx, y = y0 + ty;
  const bool valid = x < g.nx && y < g.ny;
  const int k0 = blockIdx.z * a.zchunk;
  const int k1 = min(g.nz, k0 + a.zchunk);
  const int p0 = k0 > 0 ? k0 - 1 : k0;    // first staged plane
  const int pl = k1;                      // last staged plane (zeros past the grid)

  auto stage_ptr = [&](int p) { return dsm + ((p - p0) % S) * LY::STAGE; };
  auto issue = [&](int p) {
    unsigned char* st = stage_ptr(p);
    uint64_t* bar = &bars[(p - p0) % S];
    mbar_expect_tx(bar, LY::TX_BYTES);
    tma_load_4d(st + LY::E_OFF, &maps.E, bar, x0 - 4, y0 - 1, p, 0);
    tma_load_4d(st + LY::H_OFF, &maps.H, bar, x0 - 4, y0 - 1, p, 3);
    tma_load_4d(st + LY::CB_OFF, &maps.cb, bar, x0, y0, p, 0);
  };
  bool ok = true;
  auto wait = [&](int p) {
    if (!mbar_wait(&bars[(p - p0) % S], ((p - p0) / S) & 1, kWaitCycles)) ok = false;
  };

  if (tid == 0) {
    tma_prefetch_desc(&maps.E);
    tma_prefetch_desc(&maps.H);
    tma_prefetch_desc(&maps.cb);
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int p = p0; p <= pl && p < p0 + S; ++p) issue(p);

  float hxm = 0.f, hym = 0.f;  // Ht^{n+1/2} at (x, y, k-1)
  const int xi = tx + 4, yi = ty + 1;
  if (k0 > 0) {
    wait(k0 - 1);
    wait(k0);
    if (!__syncthreads_and(ok)) goto timeout;
    if (valid) {
      const unsigned char* sc = stage_ptr(k0 - 1);
      const unsigned char* sn = stage_ptr(k0);
      float h[3];
      h_from_stage<TY>(g, reinterpret_cast<const float*>(sc + LY::E_OFF),
                       reinterpret_cast<const float*>(sn + LY::E_OFF),
                       reinterpret_cast<const float*>(sc + LY::H_OFF), xi, yi, x, y, k0 - 1, psiI,
                       nullptr, h);
      hxm = h[0];
      hym = h[1];
    }
    __syncthreads();
    if (tid == 0 && k0 - 1 + S <= pl) issue(k0 - 1 + S);
  }

  {
    double lsum = 0.0;
    for (int k = k0; k < k1; ++k) {
      if (k == k0 && k0 == 0) wait(k);
      wait(k + 1);
      if (!__syncthreads_and(ok)) goto timeout;
      const unsigned char* sc = stage_ptr(k);
      const unsigned char* sn = stage_ptr(k + 1);
      const float* Ec = reinterpret_cast<const float*>(sc + LY::E_OFF);
      const float* En = reinterpret_cast<const float*>(sn + LY::E_OFF);
      const float* Hm = reinterpret_cast<const float*>(sc + LY::H_OFF);
      const float* CB = reinterpret_cast<const float*>(sc + LY::CB_OFF);
      // Ht^{n+1/2}(k) on the tile
      float h[3] = {0.f, 0.f, 0.f};
      if (valid) {
        h_from_stage<TY>(g, Ec, En, Hm, xi, yi, x, y, k, psiI, psiO, h);
        const long long q = (long long)k * g.plane + (long long)y * g.px + x;
        Fo[3 * g.nc + q] = h[0];
        Fo[4 * g.nc + q] = h[1];
        Fo[5 * g.nc + q] = h[2];
      }
      sH[yi * W + xi] = h[0];
      sH[HP + yi * W + xi] = h[1];
      sH[2 * HP + yi * W + xi] = h[2];
      // and on the low-side ring: row y0-1 (32 cells), column x0-1 (TY+1 cells)
      for (int e = tid; e < 32 + TY + 1; e += NT) {
        int hx, hy, hi, hj;
        if (e < 32) { hx = x0 + e; hy = y0 - 1; hi = e + 4; hj = 0; }
        else { hx = x0 - 1; hy = y0 - 1 + (e - 32); hi = 3; hj = e - 32; }
        float hh[3] = {0.f, 0.f, 0.f};
        if (hx >= 0 && hy >= 0 && hx < g.nx && hy < g.ny)
          h_from_stage<TY>(g, Ec, En, Hm, hi, hj, hx, hy, k, psiI, nullptr, hh);
        sH[hj * W + hi] = hh[0];
        sH[HP + hj * W + hi] = hh[1];
        sH[2 * HP + hj * W + hi] = hh[2];
      }
      __syncthreads();
      // E^{n+1}(k) on the tile
      if (valid) {
        constexpr int EP = LY::ER * W;
        const int s0 = yi * W + xi;
        const float hx = sH[s0], hy = sH[HP + s0], hz = sH[2 * HP + s0];
        const float d6 = hz - sH[2 * HP + s0 - W];   // dHz/dy
        const float d7 = hy - hym;                   // dHy/dz
        const float d8 = hx - hxm;                   // dHx/dz
        const float d9 = hz - sH[2 * HP + s0 - 1];   // dHz/dx
        const float d10 = hy - sH[HP + s0 - 1];      // dHy/dx
        const float d11 = hx - sH[s0 - W];           // dHx/dy
        const bool sx = in_slab(x, g.nx, g.P), sy = in_slab(y, g.ny, g.P),
                   sz = in_slab(k, g.nz, g.P);
        float c0, c1, c2;
        if (!(sx || sy || sz)) {
          c0 = d6 - d7;
          c1 = d8 - d9;
          c2 = d10 - d11;
        } else {
          float t6 = d6, t7 = d7, t8 = d8, t9 = d9, t10 = d10, t11 = d11;
          if (sx) {
            t9 = cpml_t(d9, psiI, psiO, psi_x(g, 2, x, y, k), g, 0, x, PR_BE);
            t10 = cpml_t(d10, psiI, psiO, psi_x(g, 3, x, y, k), g, 0, x, PR_BE);
          }
          if (sy) {
            t6 = cpml_t(d6, psiI, psiO, psi_y(g, 2, x, y, k), g, 1, y, PR_BE);
            t11 = cpml_t(d11, psiI, psiO, psi_y(g, 3, x, y, k), g, 1, y, PR_BE);
          }
          if (sz) {
            t7 = cpml_t(d7, psiI, psiO, psi_z(g, 2, x, y, k), g, 2, k, PR_BE);
            t8 = cpml_t(d8, psiI, psiO, psi_z(g, 3, x, y, k), g, 2, k, PR_BE);
          }
          c0 = t6 - t7;
          c1 = t8 - t9;
          c2 = t10 - t11;
        }
        const float w = srcw_t(a.src, x, y, k);
        if (w != 0.f) {
          const float wj = __fmul_rn(w, a.jn);
          if (a.src.comp == 0) c0 = __fsub_rn(c0, wj);
          else if (a.src.comp == 1) c1 = __fsub_rn(c1, wj);
          else c2 = __fsub_rn(c2, wj);
        }
        const float cbv = CB[ty * 32 + tx];
        const int e0 = yi * W + xi;
        const float ex = __fadd_rn(Ec[e0], __fmul_rn(cbv, c0));
        const float ey = __fadd_rn(Ec[EP + e0], __fmul_rn(cbv, c1));
        const float ez = __fadd_rn(Ec[2 * EP + e0], __fmul_rn(cbv, c2));
        const long long q = (long long)k * g.plane + (long long)y * g.px + x;
        Fo[q] = ex;
        Fo[g.nc + q] = ey;
        Fo[2 * g.nc + q] = ez;
        int u, v;
        if (a.det.kind && on_plane(a.det.axis, a.det.index, a.det.u0, a.det.u1, a.det.v0,
                                   a.det.v1, x, y, k, &u, &v)) {
          if (a.det.kind == 1) {
            lsum += (double)ex * ex + (double)ey * ey + (double)ez * ez;
          } else {
            const float E3[3] = {ex, ey, ez}, H3[3] = {hx, hy, hz};
            const int b = (a.det.axis + 1) % 3, cc = (a.det.axis + 2) % 3;
            lsum += (double)E3[b] * H3[cc] - (double)E3[cc] * H3[b];
          }
        }
        hxm = hx;
        hym = hy;
      }
      __syncthreads();
      if (tid == 0 && k + S <= pl) issue(k + S);
    }
    if (a.det.kind) {
      double v = lsum;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0) red[tid >> 5] = v;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int wv = 0; wv < NT / 32; ++wv) t += red[wv];
        if (t != 0.0) atomicAdd(a.obj, t);
      }
    }
    return;
  }
timeout:
  if (tid == 0) {
    atomicOr(a.err, ERR_TIMEOUT);
    // let copies already in flight land before the CTA leaves
    for (int s = 0; s < S; ++s) {
      int p = -1;
      for (int q = pl; q >= p0; --q)
        if ((q - p0) % S == s) { p = q; break; }
      if (p >= 0) mbar_wait(&bars[s], ((p - p0) / S) & 1, kWaitCycles);
    }
  }
}

template <int TY, int S>
static cudaError_t launch_ft(const FwdMaps& m, const StepArgs& a, float* Fo, float* psiO,
                             cudaStream_t s) {
  const int smem = FwdLayout<TY>::bytes(S);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_fwd_tma<TY, S>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e) return e;
    attr_set = true;
  }
  dim3 grid((a.g.nx + 31) / 32, (a.g.ny + TY - 1) / TY, (a.g.nz + a.zchunk - 1) / a.zchunk);
  k_fwd_tma<TY, S><<<grid, dim3(32, TY), smem, s>>>(m, a, Fo, psiO);
  return cudaGetLastError();
}

cudaError_t launch_fwd_tma(const FwdMaps& m, const StepArgs& a, float* Fo, float* psiO,
                           cudaStream_t s) {
  switch (a.tile_y) {
    case 1: return launch_ft<1, 4>(m, a, Fo, psiO, s);
    case 2: return launch_ft<2, 4>(m, a, Fo, psiO, s);
    case 4: return launch_ft<4, 4>(m, a, Fo, psiO, s);
    case 8: return launch_ft<8, 4>(m, a, Fo, psiO, s);
    case 16: return launch_ft<16, 3>(m, a, Fo, psiO, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fdtd
