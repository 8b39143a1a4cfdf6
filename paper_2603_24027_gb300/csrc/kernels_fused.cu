// kernels_fused.cu -- fused 2.5D forward step: H and E half-steps in one pass.
//
// One CTA owns a 32 x TY column tile and marches up a z chunk.  Per plane k it
// stages E^n(k+1) (tile plus a one-cell ring) in shared memory, computes
// Ht^{n+1/2}(k) on the tile and on the low-side halo ring (x0-1, y0-1) that
// the E update's backward differences need, then E^{n+1}(k) on the tile.
// Inputs (E^n, Ht^{n-1/2}, psi) are read from one buffer and the results
// written to the other (ping-pong), so neighbouring CTAs never race and each
// cell's state is read once and written once per step (52 B/cell + CPML psi).
// The arithmetic per cell is the same sequence of rounded operations as the
// split kernels, so both paths give bit-identical fields.
#include "fdtd_internal.cuh"

namespace fdtd {

__device__ __forceinline__ float cpml_f(float d, const float* pin, float* pout, long long pi,
                                        const Geo& g, int ax, int pos, int side) {
  float b = prof(g, ax, side + 0, pos), a = prof(g, ax, side + 1, pos),
        kv = prof(g, ax, side + 2, pos);
  float s = __fmaf_rn(b, pin[pi], __fmul_rn(a, d));
  if (pout) pout[pi] = s;
  return __fmaf_rn(kv, d, s);
}

__device__ __forceinline__ double block_sum2(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int t = threadIdx.y * blockDim.x + threadIdx.x;
  int lane = t & 31, warp = t >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    int nw = (blockDim.x * blockDim.y + 31) >> 5;
    r = lane < nw ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;
}

template <int TY>
struct FwdSmem {
  float E[2][3][TY + 2][34];  // E^n planes k, k+1 on x in [x0-1, x0+33), y in [y0-1, y0+TY+1)
  float H[3][TY + 1][33];     // Ht^{n+1/2}(k) on x in [x0-1, x0+32), y in [y0-1, y0+TY)
  double red[32];
};

// Ht^{n+1/2} at (x, y, k) from the staged E planes (cur = plane k, nxt = k+1).
// ii, jj: position of (x, y) in the staged E region.
template <int TY>
__device__ __forceinline__ void h_cell(const Geo& g, const FwdSmem<TY>& sm, int cur, int nxt,
                                       int ii, int jj, int x, int y, int k, const float* Fin,
                                       const float* pin, float* pout, float h[3]) {
  const float ex = sm.E[cur][0][jj][ii], ey = sm.E[cur][1][jj][ii], ez = sm.E[cur][2][jj][ii];
  const float d0 = sm.E[cur][2][jj + 1][ii] - ez;   // dEz/dy
  const float d1 = sm.E[nxt][1][jj][ii] - ey;       // dEy/dz
  const float d2 = sm.E[nxt][0][jj][ii] - ex;       // dEx/dz
  const float d3 = sm.E[cur][2][jj][ii + 1] - ez;   // dEz/dx
  const float d4 = sm.E[cur][1][jj][ii + 1] - ey;   // dEy/dx
  const float d5 = sm.E[cur][0][jj + 1][ii] - ex;   // dEx/dy
  const bool sx = in_slab(x, g.nx, g.P), sy = in_slab(y, g.ny, g.P), sz = in_slab(k, g.nz, g.P);
  float cx, cy, cz;
  if (!(sx || sy || sz)) {
    cx = d0 - d1;
    cy = d2 - d3;
    cz = d4 - d5;
  } else {
    float t0 = d0, t1 = d1, t2 = d2, t3 = d3, t4 = d4, t5 = d5;
    if (sx) {
      t3 = cpml_f(d3, pin, pout, psi_x(g, 0, x, y, k), g, 0, x, PR_BH);
      t4 = cpml_f(d4, pin, pout, psi_x(g, 1, x, y, k), g, 0, x, PR_BH);
    }
    if (sy) {
      t0 = cpml_f(d0, pin, pout, psi_y(g, 0, x, y, k), g, 1, y, PR_BH);
      t5 = cpml_f(d5, pin, pout, psi_y(g, 1, x, y, k), g, 1, y, PR_BH);
    }
    if (sz) {
      t1 = cpml_f(d1, pin, pout, psi_z(g, 0, x, y, k), g, 2, k, PR_BH);
      t2 = cpml_f(d2, pin, pout, psi_z(g, 1, x, y, k), g, 2, k, PR_BH);
    }
    cx = t0 - t1;
    cy = t2 - t3;
    cz = t4 - t5;
  }
  const long long q = (long long)k * g.plane + (long long)y * g.px + x;
  h[0] = __fsub_rn(Fin[3 * g.nc + q], __fmul_rn(g.S, cx));
  h[1] = __fsub_rn(Fin[4 * g.nc + q], __fmul_rn(g.S, cy));
  h[2] = __fsub_rn(Fin[5 * g.nc + q], __fmul_rn(g.S, cz));
}

__device__ __forceinline__ float src_w(const Src& s, int i, int j, int k) {
  int u, v;
  if (s.kind == 0 || !on_plane(s.axis, s.index, s.u0, s.u1, s.v0, s.v1, i, j, k, &u, &v))
    return 0.f;
  return __ldg(s.w + (long long)(v - s.v0) * (s.u1 - s.u0) + (u - s.u0));
}

template <int TY>
__global__ void __launch_bounds__(32 * TY) k_fused_fwd(StepArgs a, float* __restrict__ Fo,
                                                      float* __restrict__ psiO) {
  __shared__ FwdSmem<TY> sm;
  const Geo& g = a.g;
  const float* __restrict__ Fi = a.F;
  const float* __restrict__ psiI = a.psiA;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  constexpr int NT = 32 * TY;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
  const int x = x0 + tx, y = y0 + ty;
  const bool valid = x < g.nx && y < g.ny;
  const int k0 = blockIdx.z * a.zchunk;
  const int k1 = min(g.nz, k0 + a.zchunk);

  auto load_E = [&](int b, int kk) {
    constexpr int W = 34, HH = TY + 2;
    for (int e = tid; e < W * HH; e += NT) {
      const int ii = e % W, jj = e / W;
      const int xx = x0 - 1 + ii, yy = y0 - 1 + jj;
      const bool ok = kk >= 0 && kk < g.nz && xx >= 0 && xx < g.nx && yy >= 0 && yy < g.ny;
      const long long q = (long long)kk * g.plane + (long long)yy * g.px + xx;
      sm.E[b][0][jj][ii] = ok ? Fi[q] : 0.f;
      sm.E[b][1][jj][ii] = ok ? Fi[g.nc + q] : 0.f;
      sm.E[b][2][jj][ii] = ok ? Fi[2 * g.nc + q] : 0.f;
    }
  };

  int cur = 0, nxt = 1;
  float hxm = 0.f, hym = 0.f;  // Ht^{n+1/2} at (x, y, k-1)
  if (k0 > 0) {
    load_E(cur, k0 - 1);
    load_E(nxt, k0);
    __syncthreads();
    if (valid) {
      float h[3];
      h_cell<TY>(g, sm, cur, nxt, tx + 1, ty + 1, x, y, k0 - 1, Fi, psiI, nullptr, h);
      hxm = h[0];
      hym = h[1];
    }
    __syncthreads();
    cur ^= 1;
    nxt ^= 1;
  } else {
    load_E(cur, k0);
  }

  double lsum = 0.0;
  for (int k = k0; k < k1; ++k) {
    load_E(nxt, k + 1);
    __syncthreads();
    // Ht^{n+1/2}(k) on the tile
    float h[3] = {0.f, 0.f, 0.f};
    if (valid) {
      h_cell<TY>(g, sm, cur, nxt, tx + 1, ty + 1, x, y, k, Fi, psiI, psiO, h);
      const long long q = (long long)k * g.plane + (long long)y * g.px + x;
      Fo[3 * g.nc + q] = h[0];
      Fo[4 * g.nc + q] = h[1];
      Fo[5 * g.nc + q] = h[2];
    }
    sm.H[0][ty + 1][tx + 1] = h[0];
    sm.H[1][ty + 1][tx + 1] = h[1];
    sm.H[2][ty + 1][tx + 1] = h[2];
    // ... and on the low-side halo: row y0-1 (32 cells), column x0-1 (TY+1 cells)
    for (int e = tid; e < 32 + TY + 1; e += NT) {
      int hx, hy, ii, jj;
      if (e < 32) { hx = x0 + e; hy = y0 - 1; ii = e + 1; jj = 0; }
      else { hx = x0 - 1; hy = y0 - 1 + (e - 32); ii = 0; jj = e - 32; }
      float hh[3] = {0.f, 0.f, 0.f};
      if (hx >= 0 && hy >= 0 && hx < g.nx && hy < g.ny)
        h_cell<TY>(g, sm, cur, nxt, ii, jj, hx, hy, k, Fi, psiI, nullptr, hh);
      sm.H[0][jj][ii] = hh[0];
      sm.H[1][jj][ii] = hh[1];
      sm.H[2][jj][ii] = hh[2];
    }
    __syncthreads();
    // E^{n+1}(k) on the tile
    if (valid) {
      const int ii = tx + 1, jj = ty + 1;
      const float hx = sm.H[0][jj][ii], hy = sm.H[1][jj][ii], hz = sm.H[2][jj][ii];
      const float d6 = hz - sm.H[2][jj - 1][ii];   // dHz/dy
      const float d7 = hy - hym;                   // dHy/dz
      const float d8 = hx - hxm;                   // dHx/dz
      const float d9 = hz - sm.H[2][jj][ii - 1];   // dHz/dx
      const float d10 = hy - sm.H[1][jj][ii - 1];  // dHy/dx
      const float d11 = hx - sm.H[0][jj - 1][ii];  // dHx/dy
      const bool sx = in_slab(x, g.nx, g.P), sy = in_slab(y, g.ny, g.P),
                 sz = in_slab(k, g.nz, g.P);
      float c[3];
      if (!(sx || sy || sz)) {
        c[0] = d6 - d7;
        c[1] = d8 - d9;
        c[2] = d10 - d11;
      } else {
        float t6 = d6, t7 = d7, t8 = d8, t9 = d9, t10 = d10, t11 = d11;
        if (sx) {
          t9 = cpml_f(d9, psiI, psiO, psi_x(g, 2, x, y, k), g, 0, x, PR_BE);
          t10 = cpml_f(d10, psiI, psiO, psi_x(g, 3, x, y, k), g, 0, x, PR_BE);
        }
        if (sy) {
          t6 = cpml_f(d6, psiI, psiO, psi_y(g, 2, x, y, k), g, 1, y, PR_BE);
          t11 = cpml_f(d11, psiI, psiO, psi_y(g, 3, x, y, k), g, 1, y, PR_BE);
        }
        if (sz) {
          t7 = cpml_f(d7, psiI, psiO, psi_z(g, 2, x, y, k), g, 2, k, PR_BE);
          t8 = cpml_f(d8, psiI, psiO, psi_z(g, 3, x, y, k), g, 2, k, PR_BE);
        }
        c[0] = t6 - t7;
        c[1] = t8 - t9;
        c[2] = t10 - t11;
      }
      const float w = src_w(a.src, x, y, k);
      if (w != 0.f) {
        const float wj = __fmul_rn(w, a.jn);
        if (a.src.comp == 0) c[0] = __fsub_rn(c[0], wj);
        else if (a.src.comp == 1) c[1] = __fsub_rn(c[1], wj);
        else c[2] = __fsub_rn(c[2], wj);
      }
      const long long q = (long long)k * g.plane + (long long)y * g.px + x;
      const float cbv = a.cb[q];
      const float ex = __fadd_rn(sm.E[cur][0][jj][ii], __fmul_rn(cbv, c[0]));
      const float ey = __fadd_rn(sm.E[cur][1][jj][ii], __fmul_rn(cbv, c[1]));
      const float ez = __fadd_rn(sm.E[cur][2][jj][ii], __fmul_rn(cbv, c[2]));
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
    cur ^= 1;
    nxt ^= 1;
  }
  if (a.det.kind) {
    double t = block_sum2(lsum, sm.red);
    if (tid == 0 && t != 0.0) atomicAdd(a.obj, t);
  }
}

template <int TY>
static cudaError_t launch_ff(const StepArgs& a, float* Fo, float* psiO, cudaStream_t s) {
  dim3 grid((a.g.nx + 31) / 32, (a.g.ny + TY - 1) / TY, (a.g.nz + a.zchunk - 1) / a.zchunk);
  k_fused_fwd<TY><<<grid, dim3(32, TY), 0, s>>>(a, Fo, psiO);
  return cudaGetLastError();
}

cudaError_t launch_fused_fwd(const StepArgs& a, float* Fo, float* psiO, cudaStream_t s) {
  switch (a.tile_y) {
    case 1: return launch_ff<1>(a, Fo, psiO, s);
    case 2: return launch_ff<2>(a, Fo, psiO, s);
    case 4: return launch_ff<4>(a, Fo, psiO, s);
    case 8: return launch_ff<8>(a, Fo, psiO, s);
    case 16: return launch_ff<16>(a, Fo, psiO, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused_rev(const StepArgs&, float*, float*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace fdtd
