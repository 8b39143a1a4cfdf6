// kernels_step.cu -- per-half-step Yee/CPML kernels, forward and reverse.
//
// Forward step n (Sec. 2; Yee leapfrog with convolutional PML):
//   Ht^{n+1/2} = Ht^{n-1/2} - S * curlE(E^n)               k_fwd_h
//   E^{n+1}    = E^n + cb * (curlH(Ht^{n+1/2}) - J^{n+1/2})  k_fwd_e (+ objective)
// Reverse step n (Sec. 1-2: time reversal with the interface slices injected):
//   E^n = E^{n+1} - cb * (curlH Ht^{n+1/2} - J) on the interior,
//   dL/dcb += lam_E . (curlH Ht - J),  lam_H += transpose of the E half-step   k_rev_e
//   Ht^{n-1/2} = Ht^{n+1/2} + S curlE E^n on the interior,
//   lam_E += transpose of the H half-step                                         k_rev_h
// Each kernel updates one family of arrays in place and reads only arrays it
// does not write (the adjoint psi goes through a ping-pong pair), so the
// kernels need no inter-block ordering.  Blocks are 32 x tile_y columns that
// march over a z chunk, carrying the z-neighbour plane in registers.
#include "fdtd_internal.cuh"
#include "tma.cuh"

namespace fdtd {

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    int nw = (blockDim.x * blockDim.y + 31) >> 5;
    t = lane < nw ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;
}

// kappa^-1 d + psi_new with psi_new = b psi + a d (psi updated in place).
__device__ __forceinline__ float cpml_fwd(float d, float* psi, long long pi, const Geo& g, int ax,
                                          int pos, int side) {
  float b = prof(g, ax, side + 0, pos), a = prof(g, ax, side + 1, pos),
        kv = prof(g, ax, side + 2, pos);
  float s = __fmaf_rn(b, psi[pi], __fmul_rn(a, d));  // same rounding sequence as the fused kernel
  psi[pi] = s;
  return __fmaf_rn(kv, d, s);
}

// ------------------------------------------------------------------ prep ---
__global__ void k_prep(const float* __restrict__ eps, float* __restrict__ cb, Geo g,
                       unsigned* err) {
  long long n = (long long)g.nx * g.ny * g.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % g.nx);
    long long r = t / g.nx;
    int j = (int)(r % g.ny);
    int k = (int)(r / g.ny);
    float e = eps[t];
    if (!(e >= 1.0f) || isinf(e)) {
      atomicOr(err, ERR_EPS);
      e = 1.0f;
    }
    cb[(long long)k * g.plane + (long long)j * g.px + i] = __fdiv_rn(g.S, e);
  }
}

cudaError_t launch_prep(const float* eps, float* cb, Geo g, unsigned* err, cudaStream_t s) {
  long long n = (long long)g.nx * g.ny * g.nz;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_prep<<<blocks, 256, 0, s>>>(eps, cb, g, err);
  return cudaGetLastError();
}

// -------------------------------------------------------------- fwd H ----
__global__ void __launch_bounds__(256) k_fwd_h(StepArgs a) {
  const Geo& g = a.g;
  int i = blockIdx.x * 32 + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  int k0 = blockIdx.z * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  float* __restrict__ Ex = a.F;
  float* __restrict__ Ey = a.F + g.nc;
  float* __restrict__ Ez = a.F + 2 * g.nc;
  float* __restrict__ Hx = a.F + 3 * g.nc;
  float* __restrict__ Hy = a.F + 4 * g.nc;
  float* __restrict__ Hz = a.F + 5 * g.nc;
  float* psi = a.psiA;
  const bool xn = i + 1 < g.nx, yn = j + 1 < g.ny;
  const bool sx = in_slab(i, g.nx, g.P), sy = in_slab(j, g.ny, g.P);
  long long q = (long long)k0 * g.plane + (long long)j * g.px + i;
  float ex = Ex[q], ey = Ey[q], ez = Ez[q];
  for (int k = k0; k < k1; ++k, q += g.plane) {
    const bool zn = k + 1 < g.nz;
    float ex1 = zn ? Ex[q + g.plane] : 0.f, ey1 = zn ? Ey[q + g.plane] : 0.f,
          ez1 = zn ? Ez[q + g.plane] : 0.f;
    float ezy = yn ? Ez[q + g.px] : 0.f, exy = yn ? Ex[q + g.px] : 0.f;
    float ezx = xn ? Ez[q + 1] : 0.f, eyx = xn ? Ey[q + 1] : 0.f;
    float d0 = ezy - ez, d1 = ey1 - ey, d2 = ex1 - ex, d3 = ezx - ez, d4 = eyx - ey,
          d5 = exy - ex;
    const bool sz = in_slab(k, g.nz, g.P);
    float cx, cy, cz;
    if (!(sx || sy || sz)) {
      cx = d0 - d1;
      cy = d2 - d3;
      cz = d4 - d5;
    } else {
      float t0 = d0, t1 = d1, t2 = d2, t3 = d3, t4 = d4, t5 = d5;
      if (sx) {
        t3 = cpml_fwd(d3, psi, psi_x(g, 0, i, j, k), g, 0, i, PR_BH);
        t4 = cpml_fwd(d4, psi, psi_x(g, 1, i, j, k), g, 0, i, PR_BH);
      }
      if (sy) {
        t0 = cpml_fwd(d0, psi, psi_y(g, 0, i, j, k), g, 1, j, PR_BH);
        t5 = cpml_fwd(d5, psi, psi_y(g, 1, i, j, k), g, 1, j, PR_BH);
      }
      if (sz) {
        t1 = cpml_fwd(d1, psi, psi_z(g, 0, i, j, k), g, 2, k, PR_BH);
        t2 = cpml_fwd(d2, psi, psi_z(g, 1, i, j, k), g, 2, k, PR_BH);
      }
      cx = t0 - t1;
      cy = t2 - t3;
      cz = t4 - t5;
    }
    Hx[q] = __fsub_rn(Hx[q], __fmul_rn(g.S, cx));
    Hy[q] = __fsub_rn(Hy[q], __fmul_rn(g.S, cy));
    Hz[q] = __fsub_rn(Hz[q], __fmul_rn(g.S, cz));
    ex = ex1;
    ey = ey1;
    ez = ez1;
  }
}

// Split kernels are built for at most 256 threads: tile heights above 8 run as 8.
static int split_ty(const StepArgs& a) { return a.tile_y > 8 ? 8 : a.tile_y; }

static dim3 step_grid(const StepArgs& a) {
  int ty = split_ty(a);
  int zc = a.zchunk;
  return dim3((a.g.nx + 31) / 32, (a.g.ny + ty - 1) / ty, (a.g.nz + zc - 1) / zc);
}

cudaError_t launch_fwd_h(const StepArgs& a, cudaStream_t s) {
  k_fwd_h<<<step_grid(a), dim3(32, split_ty(a)), 0, s>>>(a);
  return cudaGetLastError();
}

// -------------------------------------------------------------- fwd E ----
__device__ __forceinline__ float src_weight(const Src& s, int i, int j, int k) {
  int u, v;
  if (s.kind == 0 || !on_plane(s.axis, s.index, s.u0, s.u1, s.v0, s.v1, i, j, k, &u, &v))
    return 0.f;
  return __ldg(s.w + (long long)(v - s.v0) * (s.u1 - s.u0) + (u - s.u0));
}

__device__ __forceinline__ double det_value(const Det& d, float ex, float ey, float ez, float hx,
                                            float hy, float hz) {
  if (d.kind == 1) return (double)ex * ex + (double)ey * ey + (double)ez * ez;
  float E[3] = {ex, ey, ez}, H[3] = {hx, hy, hz};
  int b = (d.axis + 1) % 3, c = (d.axis + 2) % 3;
  return (double)E[b] * H[c] - (double)E[c] * H[b];
}

__global__ void __launch_bounds__(256) k_fwd_e(StepArgs a) {
  __shared__ double sh[32];
  const Geo& g = a.g;
  int i = blockIdx.x * 32 + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  double lsum = 0.0;
  if (i < g.nx && j < g.ny) {
    int k0 = blockIdx.z * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
    float* __restrict__ Ex = a.F;
    float* __restrict__ Ey = a.F + g.nc;
    float* __restrict__ Ez = a.F + 2 * g.nc;
    const float* __restrict__ Hx = a.F + 3 * g.nc;
    const float* __restrict__ Hy = a.F + 4 * g.nc;
    const float* __restrict__ Hz = a.F + 5 * g.nc;
    float* psi = a.psiA;
    const bool xp = i > 0, yp = j > 0;
    const bool sx = in_slab(i, g.nx, g.P), sy = in_slab(j, g.ny, g.P);
    long long q = (long long)k0 * g.plane + (long long)j * g.px + i;
    float hxm = k0 > 0 ? Hx[q - g.plane] : 0.f, hym = k0 > 0 ? Hy[q - g.plane] : 0.f;
    for (int k = k0; k < k1; ++k, q += g.plane) {
      float hx = Hx[q], hy = Hy[q], hz = Hz[q];
      float hzy = yp ? Hz[q - g.px] : 0.f, hxy = yp ? Hx[q - g.px] : 0.f;
      float hzx = xp ? Hz[q - 1] : 0.f, hyx = xp ? Hy[q - 1] : 0.f;
      float d6 = hz - hzy, d7 = hy - hym, d8 = hx - hxm, d9 = hz - hzx, d10 = hy - hyx,
            d11 = hx - hxy;
      const bool sz = in_slab(k, g.nz, g.P);
      float c[3];
      if (!(sx || sy || sz)) {
        c[0] = d6 - d7;
        c[1] = d8 - d9;
        c[2] = d10 - d11;
      } else {
        float t6 = d6, t7 = d7, t8 = d8, t9 = d9, t10 = d10, t11 = d11;
        if (sx) {
          t9 = cpml_fwd(d9, psi, psi_x(g, 2, i, j, k), g, 0, i, PR_BE);
          t10 = cpml_fwd(d10, psi, psi_x(g, 3, i, j, k), g, 0, i, PR_BE);
        }
        if (sy) {
          t6 = cpml_fwd(d6, psi, psi_y(g, 2, i, j, k), g, 1, j, PR_BE);
          t11 = cpml_fwd(d11, psi, psi_y(g, 3, i, j, k), g, 1, j, PR_BE);
        }
        if (sz) {
          t7 = cpml_fwd(d7, psi, psi_z(g, 2, i, j, k), g, 2, k, PR_BE);
          t8 = cpml_fwd(d8, psi, psi_z(g, 3, i, j, k), g, 2, k, PR_BE);
        }
        c[0] = t6 - t7;
        c[1] = t8 - t9;
        c[2] = t10 - t11;
      }
      float w = src_weight(a.src, i, j, k);
      if (w != 0.f) c[a.src.comp] = __fsub_rn(c[a.src.comp], __fmul_rn(w, a.jn));
      float cbv = a.cb[q];
      float ex = __fadd_rn(Ex[q], __fmul_rn(cbv, c[0]));
      float ey = __fadd_rn(Ey[q], __fmul_rn(cbv, c[1]));
      float ez = __fadd_rn(Ez[q], __fmul_rn(cbv, c[2]));
      Ex[q] = ex;
      Ey[q] = ey;
      Ez[q] = ez;
      int u, v;
      if (a.det.kind && on_plane(a.det.axis, a.det.index, a.det.u0, a.det.u1, a.det.v0, a.det.v1,
                                 i, j, k, &u, &v))
        lsum += det_value(a.det, ex, ey, ez, hx, hy, hz);
      hxm = hx;
      hym = hy;
    }
  }
  if (a.det.kind) {
    double t = block_sum(lsum, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0 && t != 0.0) atomicAdd(a.obj, t);
  }
}

cudaError_t launch_fwd_e(const StepArgs& a, cudaStream_t s) {
  k_fwd_e<<<step_grid(a), dim3(32, split_ty(a)), 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------- reverse ---
// Adjoint difference term of one CPML curl term at a cell:
//   v = coefficient * lambda_field at that cell,
//   slab:   mu = lam_psi + v,  return kinv v + a mu   (and lam_psi_new = b mu)
//   else:   return v.
__device__ __forceinline__ float adj_term(float v, const float* lpA, float* lpB, long long pi,
                                          const Geo& g, int ax, int pos, int side, bool own) {
  int n = ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz);
  if (!in_slab(pos, n, g.P)) return v;
  float mu = lpA[pi] + v;
  if (own) lpB[pi] = prof(g, ax, side + 0, pos) * mu;
  return prof(g, ax, side + 2, pos) * v + prof(g, ax, side + 1, pos) * mu;
}

__device__ __forceinline__ bool interior(const Geo& g, int i, int j, int k) {
  return i >= g.P && i < g.nx - g.P && j >= g.P && j < g.ny - g.P && k >= g.P && k < g.nz - g.P;
}

__global__ void __launch_bounds__(256) k_rev_e(StepArgs a) {
  const Geo& g = a.g;
  int i = blockIdx.x * 32 + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  int k0 = blockIdx.z * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  float* __restrict__ Ex = a.F;
  float* __restrict__ Ey = a.F + g.nc;
  float* __restrict__ Ez = a.F + 2 * g.nc;
  const float* __restrict__ Hx = a.F + 3 * g.nc;
  const float* __restrict__ Hy = a.F + 4 * g.nc;
  const float* __restrict__ Hz = a.F + 5 * g.nc;
  const float* __restrict__ lEx = a.L;
  const float* __restrict__ lEy = a.L + g.nc;
  const float* __restrict__ lEz = a.L + 2 * g.nc;
  float* __restrict__ lHx = a.L + 3 * g.nc;
  float* __restrict__ lHy = a.L + 4 * g.nc;
  float* __restrict__ lHz = a.L + 5 * g.nc;
  const float* lpA = a.psiA;
  float* lpB = a.psiB;
  const float* __restrict__ cb = a.cb;
  const bool xn = i + 1 < g.nx, yn = j + 1 < g.ny;
  const int dX = a.dhi[0] - a.dlo[0], dY = a.dhi[1] - a.dlo[1];
  long long q = (long long)k0 * g.plane + (long long)j * g.px + i;
  for (int k = k0; k < k1; ++k, q += g.plane) {
    float cbv = cb[q];
    float lex = lEx[q], ley = lEy[q], lez = lEz[q];
    // primal inverse E update on the interior + dL/dcb
    if (interior(g, i, j, k)) {
      float hx = Hx[q], hy = Hy[q], hz = Hz[q];
      float d6 = hz - Hz[q - g.px], d7 = hy - Hy[q - g.plane], d8 = hx - Hx[q - g.plane];
      float d9 = hz - Hz[q - 1], d10 = hy - Hy[q - 1], d11 = hx - Hx[q - g.px];
      float c[3] = {d6 - d7, d8 - d9, d10 - d11};
      float w = src_weight(a.src, i, j, k);
      if (w != 0.f) c[a.src.comp] = __fsub_rn(c[a.src.comp], __fmul_rn(w, a.jn));
      Ex[q] = __fsub_rn(Ex[q], __fmul_rn(cbv, c[0]));
      Ey[q] = __fsub_rn(Ey[q], __fmul_rn(cbv, c[1]));
      Ez[q] = __fsub_rn(Ez[q], __fmul_rn(cbv, c[2]));
      if (i >= a.dlo[0] && i < a.dhi[0] && j >= a.dlo[1] && j < a.dhi[1] && k >= a.dlo[2] &&
          k < a.dhi[2]) {
        float s = lex * c[0] + ley * c[1] + lez * c[2];
        long long qd = ((long long)(k - a.dlo[2]) * dY + (j - a.dlo[1])) * dX + (i - a.dlo[0]);
        a.gacc[qd] += (double)s;
      }
    }
    // adjoint of the E half-step: lam_H += D'^T lam_delta'
    float wx = cbv * lex, wy = cbv * ley, wz = cbv * lez;
    // own-cell terms (t6: Ex,y,+ ; t7: Ex,z,- ; t8: Ey,z,+ ; t9: Ey,x,- ; t10: Ez,x,+ ; t11: Ez,y,-)
    float o6 = adj_term(wx, lpA, lpB, psi_y(g, 2, i, j, k), g, 1, j, PR_BE, true);
    float o11 = adj_term(-wz, lpA, lpB, psi_y(g, 3, i, j, k), g, 1, j, PR_BE, true);
    float o7 = adj_term(-wx, lpA, lpB, psi_z(g, 2, i, j, k), g, 2, k, PR_BE, true);
    float o8 = adj_term(wy, lpA, lpB, psi_z(g, 3, i, j, k), g, 2, k, PR_BE, true);
    float o9 = adj_term(-wy, lpA, lpB, psi_x(g, 2, i, j, k), g, 0, i, PR_BE, true);
    float o10 = adj_term(wz, lpA, lpB, psi_x(g, 3, i, j, k), g, 0, i, PR_BE, true);
    // neighbour terms
    float n6 = 0.f, n11 = 0.f, n7 = 0.f, n8 = 0.f, n9 = 0.f, n10 = 0.f;
    if (yn) {
      long long r = q + g.px;
      float c2 = cb[r];
      n6 = adj_term(c2 * lEx[r], lpA, lpB, psi_y(g, 2, i, j + 1, k), g, 1, j + 1, PR_BE, false);
      n11 = adj_term(-c2 * lEz[r], lpA, lpB, psi_y(g, 3, i, j + 1, k), g, 1, j + 1, PR_BE, false);
    }
    if (k + 1 < g.nz) {
      long long r = q + g.plane;
      float c2 = cb[r];
      n7 = adj_term(-c2 * lEx[r], lpA, lpB, psi_z(g, 2, i, j, k + 1), g, 2, k + 1, PR_BE, false);
      n8 = adj_term(c2 * lEy[r], lpA, lpB, psi_z(g, 3, i, j, k + 1), g, 2, k + 1, PR_BE, false);
    }
    if (xn) {
      long long r = q + 1;
      float c2 = cb[r];
      n9 = adj_term(-c2 * lEy[r], lpA, lpB, psi_x(g, 2, i + 1, j, k), g, 0, i + 1, PR_BE, false);
      n10 = adj_term(c2 * lEz[r], lpA, lpB, psi_x(g, 3, i + 1, j, k), g, 0, i + 1, PR_BE, false);
    }
    lHx[q] += (o8 - n8) + (o11 - n11);
    lHy[q] += (o7 - n7) + (o10 - n10);
    lHz[q] += (o6 - n6) + (o9 - n9);
  }
}

cudaError_t launch_rev_e(const StepArgs& a, cudaStream_t s) {
  k_rev_e<<<step_grid(a), dim3(32, split_ty(a)), 0, s>>>(a);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_rev_h(StepArgs a) {
  const Geo& g = a.g;
  int i = blockIdx.x * 32 + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  int k0 = blockIdx.z * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  const float* __restrict__ Ex = a.F;
  const float* __restrict__ Ey = a.F + g.nc;
  const float* __restrict__ Ez = a.F + 2 * g.nc;
  float* __restrict__ Hx = a.F + 3 * g.nc;
  float* __restrict__ Hy = a.F + 4 * g.nc;
  float* __restrict__ Hz = a.F + 5 * g.nc;
  float* __restrict__ lEx = a.L;
  float* __restrict__ lEy = a.L + g.nc;
  float* __restrict__ lEz = a.L + 2 * g.nc;
  const float* __restrict__ lHx = a.L + 3 * g.nc;
  const float* __restrict__ lHy = a.L + 4 * g.nc;
  const float* __restrict__ lHz = a.L + 5 * g.nc;
  const float* lpA = a.psiA;
  float* lpB = a.psiB;
  const float S = g.S;
  long long q = (long long)k0 * g.plane + (long long)j * g.px + i;
  for (int k = k0; k < k1; ++k, q += g.plane) {
    // primal inverse H update on the interior
    if (interior(g, i, j, k)) {
      float ex = Ex[q], ey = Ey[q], ez = Ez[q];
      float d0 = Ez[q + g.px] - ez, d1 = Ey[q + g.plane] - ey, d2 = Ex[q + g.plane] - ex;
      float d3 = Ez[q + 1] - ez, d4 = Ey[q + 1] - ey, d5 = Ex[q + g.px] - ex;
      Hx[q] = __fadd_rn(Hx[q], __fmul_rn(S, d0 - d1));
      Hy[q] = __fadd_rn(Hy[q], __fmul_rn(S, d2 - d3));
      Hz[q] = __fadd_rn(Hz[q], __fmul_rn(S, d4 - d5));
    }
    // adjoint of the H half-step: lam_E += D^T lam_delta, v = -S s lam_H
    // terms t0: Hx,y,+ ; t1: Hx,z,- ; t2: Hy,z,+ ; t3: Hy,x,- ; t4: Hz,x,+ ; t5: Hz,y,-
    float lhx = lHx[q], lhy = lHy[q], lhz = lHz[q];
    float o0 = adj_term(-S * lhx, lpA, lpB, psi_y(g, 0, i, j, k), g, 1, j, PR_BH, true);
    float o5 = adj_term(S * lhz, lpA, lpB, psi_y(g, 1, i, j, k), g, 1, j, PR_BH, true);
    float o1 = adj_term(S * lhx, lpA, lpB, psi_z(g, 0, i, j, k), g, 2, k, PR_BH, true);
    float o2 = adj_term(-S * lhy, lpA, lpB, psi_z(g, 1, i, j, k), g, 2, k, PR_BH, true);
    float o3 = adj_term(S * lhy, lpA, lpB, psi_x(g, 0, i, j, k), g, 0, i, PR_BH, true);
    float o4 = adj_term(-S * lhz, lpA, lpB, psi_x(g, 1, i, j, k), g, 0, i, PR_BH, true);
    float m0 = 0.f, m5 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
    if (j > 0) {
      long long r = q - g.px;
      m0 = adj_term(-S * lHx[r], lpA, lpB, psi_y(g, 0, i, j - 1, k), g, 1, j - 1, PR_BH, false);
      m5 = adj_term(S * lHz[r], lpA, lpB, psi_y(g, 1, i, j - 1, k), g, 1, j - 1, PR_BH, false);
    }
    if (k > 0) {
      long long r = q - g.plane;
      m1 = adj_term(S * lHx[r], lpA, lpB, psi_z(g, 0, i, j, k - 1), g, 2, k - 1, PR_BH, false);
      m2 = adj_term(-S * lHy[r], lpA, lpB, psi_z(g, 1, i, j, k - 1), g, 2, k - 1, PR_BH, false);
    }
    if (i > 0) {
      long long r = q - 1;
      m3 = adj_term(S * lHy[r], lpA, lpB, psi_x(g, 0, i - 1, j, k), g, 0, i - 1, PR_BH, false);
      m4 = adj_term(-S * lHz[r], lpA, lpB, psi_x(g, 1, i - 1, j, k), g, 0, i - 1, PR_BH, false);
    }
    lEx[q] += (m2 - o2) + (m5 - o5);
    lEy[q] += (m1 - o1) + (m4 - o4);
    lEz[q] += (m0 - o0) + (m3 - o3);
  }
}

cudaError_t launch_rev_h(const StepArgs& a, cudaStream_t s) {
  k_rev_h<<<step_grid(a), dim3(32, split_ty(a)), 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------ finalize ---
// dL/d(eps) = -(cb / eps) sum_n lam_E . X = -(cb^2 / S) * acc, times the seed.
__global__ void k_finalize(const double* __restrict__ gacc, const float* __restrict__ cb, Geo g,
                           int x0, int y0, int z0, int dX, int dY, int dZ, double scale,
                           float* __restrict__ out, unsigned* err) {
  long long n = (long long)dX * dY * dZ;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % dX);
    long long r = t / dX;
    int j = (int)(r % dY);
    int k = (int)(r / dY);
    double c = cb[(long long)(k + z0) * g.plane + (long long)(j + y0) * g.px + (i + x0)];
    double v = -scale * c * c / (double)g.S * gacc[t];
    if (!isfinite(v)) atomicOr(err, ERR_NONFINITE);
    out[t] = (float)v;
  }
}

cudaError_t launch_finalize(const double* gacc, const float* cb, Geo g, const int* dlo,
                            const int* dhi, double scale, float* out, unsigned* err,
                            cudaStream_t s) {
  int dX = dhi[0] - dlo[0], dY = dhi[1] - dlo[1], dZ = dhi[2] - dlo[2];
  long long n = (long long)dX * dY * dZ;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  k_finalize<<<blocks, 256, 0, s>>>(gacc, cb, g, dlo[0], dlo[1], dlo[2], dX, dY, dZ, scale, out,
                                    err);
  return cudaGetLastError();
}

// -------------------------------------------------------- wait self-test ---
// An mbarrier armed for 16 transaction bytes that no copy delivers: the
// bounded wait of the TMA pipelines must give up and report.
__global__ void k_wait_selftest(long long limit, unsigned* flag) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, 16);
    if (!mbar_wait(&bar, 0, limit)) atomicOr(flag, ERR_TIMEOUT);
  }
}

cudaError_t launch_wait_selftest(long long limit, unsigned* flag, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(limit, flag);
  return cudaGetLastError();
}

// -------------------------------------------------------------- monitor ---
// Objective l_n of a detector plane from (E^{n+1}, Ht^{n+1/2}) in F: one
// thread per plane cell, FP64 block sums, one atomic per block into *out.
__global__ void __launch_bounds__(256) k_monitor(const float* __restrict__ F, Geo g, Det d,
                                                 double* out) {
  __shared__ double red[8];
  const int du = d.u1 - d.u0, dv = d.v1 - d.v0;
  const int r = blockIdx.x * 256 + threadIdx.x;
  double v = 0.0;
  if (r < du * dv) {
    const int vv = r / du, uu = r - vv * du;
    const int u = d.u0 + uu, w = d.v0 + vv;
    const int x = d.axis == 0 ? d.index : u;
    const int y = d.axis == 1 ? d.index : (d.axis == 0 ? u : w);
    const int z = d.axis == 2 ? d.index : w;
    const long long q = (long long)z * g.plane + (long long)y * g.px + x;
    if (d.kind == 1) {
      for (int c = 0; c < 3; ++c) {
        const double e = F[c * g.nc + q];
        v += e * e;
      }
    } else {
      const int b = (d.axis + 1) % 3, c = (d.axis + 2) % 3;
      v = (double)F[b * g.nc + q] * F[(3 + c) * g.nc + q] -
          (double)F[c * g.nc + q] * F[(3 + b) * g.nc + q];
    }
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    if (t != 0.0) atomicAdd(out, t);
  }
}

cudaError_t launch_monitor(const float* F, Geo g, const Det& d, double* out, cudaStream_t s) {
  const int n = (d.u1 - d.u0) * (d.v1 - d.v0);
  k_monitor<<<(n + 255) / 256, 256, 0, s>>>(F, g, d, out);
  return cudaGetLastError();
}

// --------------------------------------------------------------- gather ---
__global__ void k_gather(const float* __restrict__ F, Geo g, float* __restrict__ out) {
  long long n = (long long)g.nx * g.ny * g.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 6 * n;
       t += (long long)gridDim.x * blockDim.x) {
    int c = (int)(t / n);
    long long r = t % n;
    int i = (int)(r % g.nx);
    long long r2 = r / g.nx;
    int j = (int)(r2 % g.ny);
    int k = (int)(r2 / g.ny);
    out[t] = F[c * g.nc + (long long)k * g.plane + (long long)j * g.px + i];
  }
}

cudaError_t launch_gather(const float* F, Geo g, float* out, cudaStream_t s) {
  k_gather<<<152 * 8, 256, 0, s>>>(F, g, out);
  return cudaGetLastError();
}

}  // namespace fdtd
