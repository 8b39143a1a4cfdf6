// kernels_lag.cu -- TMA half-step kernels that read one plane per iteration.
//
// The same four half-steps as kernels_split_tma.cu, restructured so that an
// iteration only touches the plane it has just received: the z-neighbour
// values a cell needs from the plane below are carried in registers from the
// previous iteration, and the parts of an update that need the plane above
// are finished one iteration later (the update of plane p-1 completes while
// plane p is resident).  A stage therefore never has to outlive its own
// iteration: an S-stage ring keeps S-1 planes in flight, and the boxes cover
// exactly the neighbours each kernel reads (36 x (TY+1) instead of a full
// ring), which leaves room for more CTAs per SM.  Arithmetic per cell is the
// same sequence of rounded operations as the other kernel variants,
// including the association of every sum, so results are bit-identical.
#include <cudaTypedefs.h>

#include "lag_common.cuh"

namespace fdtd {

// =================================================== forward H half-step ===
template <int TY, int S>
__global__ void __launch_bounds__(32 * TY) k_lfwd_h(const __grid_constant__ LagMaps m,
                                                   StepArgs a) {
  typedef G<TY> B;
  typedef LFH<TY, S> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
  const int x = x0 + tx, y = y0 + ty;
  const bool valid = x < g.nx && y < g.ny;
  const int k0 = blockIdx.z * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  const bool txs = tile_in_slab(x0, min(x0 + 31, g.nx - 1), g.nx, g.P);
  const bool tys = tile_in_slab(y0, min(y0 + TY - 1, g.ny - 1), g.ny, g.P);
  // plane p < k1 starts Ht(p); plane p > k0 finishes Ht(p-1) (needs E(p))
  Ring<S> R = ring_setup<S>(dsm, Y::STAGE, k0, k1);
  auto issue = [&](int p) {
    unsigned char* st = R.at(p);
    uint64_t* bar = R.bar(p);
    const bool body = p < k1;
    const bool zs = body && in_slab(p, g.nz, g.P);
    uint32_t bytes = 3 * B::P * 4 + (body ? 3 * B::OP * 4 : 0) + (body && txs ? 2 * B::OP * 4 : 0) +
                     (body && tys ? 2 * B::OP * 4 : 0) + (zs ? 2 * B::OP * 4 : 0);
    mbar_expect_tx(bar, bytes);
    tma_load_4d(st + Y::E, &m.Fw, bar, x0, y0, p, 0);
    if (body) tma_load_4d(st + Y::H, &m.Fo, bar, x0, y0, p, 3);
    if (body && txs) tma_load_4d(st + Y::PX, &m.Po, bar, x0, y0, p, 0);
    if (body && tys) tma_load_4d(st + Y::PY, &m.Po, bar, x0, y0, p, 4);
    if (zs) tma_load_4d(st + Y::PZ, &m.Po, bar, x0, y0, p, 8);
  };
  if (tid == 0)
    for (int p = R.p0; p <= R.p1 && p < R.p0 + S; ++p) issue(p);
  const bool sx = valid && in_slab(x, g.nx, g.P), sy = valid && in_slab(y, g.ny, g.P);
  float bx = 0.f, ax = 0.f, kx = 1.f, by = 0.f, ay = 0.f, ky = 1.f;
  if (sx) { bx = prof(g, 0, PR_BH, x); ax = prof(g, 0, PR_AH, x); kx = prof(g, 0, PR_KH, x); }
  if (sy) { by = prof(g, 1, PR_BH, y); ay = prof(g, 1, PR_AH, y); ky = prof(g, 1, PR_KH, y); }
  const int hb = ty * B::W + tx;   // own cell in a hi box
  const int ob = ty * 32 + tx;     // own cell in an own box
  const long long nc = g.nc;
  float* F = a.F;
  float* psi = a.psiA;
  long long q = (long long)k0 * g.plane + (long long)y * g.px + x;   // plane of the carried cell
  // carried state of Ht(p-1)
  float c_ex = 0.f, c_ey = 0.f, c_t0 = 0.f, c_t3 = 0.f, c_t4 = 0.f, c_t5 = 0.f;
  float c_hx = 0.f, c_hy = 0.f, c_hz = 0.f, c_pz0 = 0.f, c_pz1 = 0.f;
  bool ok = true;
  for (int p = k0; p <= k1; ++p) {
    if (!R.wait(p)) ok = false;
    if (!__syncthreads_and(ok)) { ring_drain<S>(R, p, a.err); return; }
    const unsigned char* st = R.at(p);
    const float* Eb = reinterpret_cast<const float*>(st + Y::E);
    if (valid) {
      if (p > k0) {  // finish Ht(p-1) with dEy/dz and dEx/dz
        const int k = p - 1;
        const float d1 = Eb[B::P + hb] - c_ey;
        const float d2 = Eb[hb] - c_ex;
        float t1 = d1, t2 = d2;
        if (in_slab(k, g.nz, g.P)) {
          const float bz = prof(g, 2, PR_BH, k), az = prof(g, 2, PR_AH, k), kz = prof(g, 2, PR_KH, k);
          t1 = cpml_s(d1, c_pz0, psi, 8 * nc + q, bz, az, kz);
          t2 = cpml_s(d2, c_pz1, psi, 9 * nc + q, bz, az, kz);
        }
        const float cx = c_t0 - t1, cy = t2 - c_t3, cz = c_t4 - c_t5;
        F[3 * nc + q] = __fsub_rn(c_hx, __fmul_rn(g.S, cx));
        F[4 * nc + q] = __fsub_rn(c_hy, __fmul_rn(g.S, cy));
        F[5 * nc + q] = __fsub_rn(c_hz, __fmul_rn(g.S, cz));
        q += g.plane;
      }
      if (p < k1) {  // start Ht(p): x and y derivatives, their psi updates
        const float ex = Eb[hb], ey = Eb[B::P + hb], ez = Eb[2 * B::P + hb];
        float t0 = Eb[2 * B::P + hb + B::W] - ez;   // dEz/dy
        float t3 = Eb[2 * B::P + hb + 1] - ez;      // dEz/dx
        float t4 = Eb[B::P + hb + 1] - ey;          // dEy/dx
        float t5 = Eb[hb + B::W] - ex;              // dEx/dy
        if (sx) {
          const float* P = reinterpret_cast<const float*>(st + Y::PX);
          t3 = cpml_s(t3, P[ob], psi, 0 * nc + q, bx, ax, kx);
          t4 = cpml_s(t4, P[B::OP + ob], psi, 1 * nc + q, bx, ax, kx);
        }
        if (sy) {
          const float* P = reinterpret_cast<const float*>(st + Y::PY);
          t0 = cpml_s(t0, P[ob], psi, 4 * nc + q, by, ay, ky);
          t5 = cpml_s(t5, P[B::OP + ob], psi, 5 * nc + q, by, ay, ky);
        }
        const float* Ho = reinterpret_cast<const float*>(st + Y::H);
        c_ex = ex; c_ey = ey; c_t0 = t0; c_t3 = t3; c_t4 = t4; c_t5 = t5;
        c_hx = Ho[ob]; c_hy = Ho[B::OP + ob]; c_hz = Ho[2 * B::OP + ob];
        if (in_slab(p, g.nz, g.P)) {
          const float* P = reinterpret_cast<const float*>(st + Y::PZ);
          c_pz0 = P[ob];
          c_pz1 = P[B::OP + ob];
        }
      }
    }
    __syncthreads();
    if (tid == 0 && p + S <= R.p1) issue(p + S);
  }
}

// =================================================== forward E half-step ===

template <int TY, int S>
__global__ void __launch_bounds__(32 * TY) k_lfwd_e(const __grid_constant__ LagMaps m,
                                                   StepArgs a) {
  typedef G<TY> B;
  typedef LFE<TY, S> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
  const int x = x0 + tx, y = y0 + ty;
  const bool valid = x < g.nx && y < g.ny;
  const int k0 = blockIdx.z * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  const bool txs = tile_in_slab(x0, min(x0 + 31, g.nx - 1), g.nx, g.P);
  const bool tys = tile_in_slab(y0, min(y0 + TY - 1, g.ny - 1), g.ny, g.P);
  // plane k0-1 only provides Ht(k0-1) at the own cell
  Ring<S> R = ring_setup<S>(dsm, Y::STAGE, k0 - 1, k1 - 1);
  double* red = reinterpret_cast<double*>(dsm + S * Y::STAGE + 8 * S + 64);
  auto issue = [&](int p) {
    unsigned char* st = R.at(p);
    uint64_t* bar = R.bar(p);
    const bool body = p >= k0;
    const bool zs = body && in_slab(p, g.nz, g.P);
    uint32_t bytes = 3 * B::P * 4 + (body ? 4 * B::OP * 4 : 0) + (body && txs ? 2 * B::OP * 4 : 0) +
                     (body && tys ? 2 * B::OP * 4 : 0) + (zs ? 2 * B::OP * 4 : 0);
    mbar_expect_tx(bar, bytes);
    tma_load_4d(st + Y::H, &m.Fw, bar, x0 - 4, y0 - 1, p, 3);
    if (body) {
      tma_load_4d(st + Y::E, &m.Fo, bar, x0, y0, p, 0);
      tma_load_4d(st + Y::CB, &m.cbo, bar, x0, y0, p, 0);
    }
    if (body && txs) tma_load_4d(st + Y::PX, &m.Po, bar, x0, y0, p, 2);
    if (body && tys) tma_load_4d(st + Y::PY, &m.Po, bar, x0, y0, p, 6);
    if (zs) tma_load_4d(st + Y::PZ, &m.Po, bar, x0, y0, p, 10);
  };
  if (tid == 0)
    for (int p = R.p0; p <= R.p1 && p < R.p0 + S; ++p) issue(p);
  const bool sx = valid && in_slab(x, g.nx, g.P), sy = valid && in_slab(y, g.ny, g.P);
  float bx = 0.f, ax = 0.f, kx = 1.f, by = 0.f, ay = 0.f, ky = 1.f;
  if (sx) { bx = prof(g, 0, PR_BE, x); ax = prof(g, 0, PR_AE, x); kx = prof(g, 0, PR_KE, x); }
  if (sy) { by = prof(g, 1, PR_BE, y); ay = prof(g, 1, PR_AE, y); ky = prof(g, 1, PR_KE, y); }
  const int lb = (ty + 1) * B::W + tx + 4;   // own cell in a lo box
  const int ob = ty * 32 + tx;
  const long long nc = g.nc;
  float* F = a.F;
  float* psi = a.psiA;
  long long q = (long long)k0 * g.plane + (long long)y * g.px + x;
  float c_hx = 0.f, c_hy = 0.f;   // Ht(p-1) at the own cell
  double lsum = 0.0;
  bool ok = true;
  for (int p = k0 - 1; p < k1; ++p) {
    if (!R.wait(p)) ok = false;
    if (!__syncthreads_and(ok)) { ring_drain<S>(R, p, a.err); return; }
    const unsigned char* st = R.at(p);
    const float* Hb = reinterpret_cast<const float*>(st + Y::H);
    if (valid) {
      const float hx = Hb[lb], hy = Hb[B::P + lb], hz = Hb[2 * B::P + lb];
      if (p >= k0) {
        const int k = p;
        const float d6 = hz - Hb[2 * B::P + lb - B::W];   // dHz/dy
        const float d7 = hy - c_hy;                       // dHy/dz
        const float d8 = hx - c_hx;                       // dHx/dz
        const float d9 = hz - Hb[2 * B::P + lb - 1];      // dHz/dx
        const float d10 = hy - Hb[B::P + lb - 1];         // dHy/dx
        const float d11 = hx - Hb[lb - B::W];             // dHx/dy
        const bool sz = in_slab(k, g.nz, g.P);
        float c0, c1, c2;
        if (!(sx || sy || sz)) {
          c0 = d6 - d7;
          c1 = d8 - d9;
          c2 = d10 - d11;
        } else {
          float t6 = d6, t7 = d7, t8 = d8, t9 = d9, t10 = d10, t11 = d11;
          if (sx) {
            const float* P = reinterpret_cast<const float*>(st + Y::PX);
            t9 = cpml_s(d9, P[ob], psi, 2 * nc + q, bx, ax, kx);
            t10 = cpml_s(d10, P[B::OP + ob], psi, 3 * nc + q, bx, ax, kx);
          }
          if (sy) {
            const float* P = reinterpret_cast<const float*>(st + Y::PY);
            t6 = cpml_s(d6, P[ob], psi, 6 * nc + q, by, ay, ky);
            t11 = cpml_s(d11, P[B::OP + ob], psi, 7 * nc + q, by, ay, ky);
          }
          if (sz) {
            const float* P = reinterpret_cast<const float*>(st + Y::PZ);
            const float bz = prof(g, 2, PR_BE, k), az = prof(g, 2, PR_AE, k), kz = prof(g, 2, PR_KE, k);
            t7 = cpml_s(d7, P[ob], psi, 10 * nc + q, bz, az, kz);
            t8 = cpml_s(d8, P[B::OP + ob], psi, 11 * nc + q, bz, az, kz);
          }
          c0 = t6 - t7;
          c1 = t8 - t9;
          c2 = t10 - t11;
        }
        if (a.src.kind) {
          const float w = src_wt(a.src, x, y, k);
          if (w != 0.f) {
            const float wj = __fmul_rn(w, a.jn);
            if (a.src.comp == 0) c0 = __fsub_rn(c0, wj);
            else if (a.src.comp == 1) c1 = __fsub_rn(c1, wj);
            else c2 = __fsub_rn(c2, wj);
          }
        }
        const float* Eo = reinterpret_cast<const float*>(st + Y::E);
        const float cbv = reinterpret_cast<const float*>(st + Y::CB)[ob];
        const float ex = __fadd_rn(Eo[ob], __fmul_rn(cbv, c0));
        const float ey = __fadd_rn(Eo[B::OP + ob], __fmul_rn(cbv, c1));
        const float ez = __fadd_rn(Eo[2 * B::OP + ob], __fmul_rn(cbv, c2));
        F[q] = ex;
        F[nc + q] = ey;
        F[2 * nc + q] = ez;
        int u, v;
        if (a.det.kind && on_plane(a.det.axis, a.det.index, a.det.u0, a.det.u1, a.det.v0,
                                   a.det.v1, x, y, k, &u, &v)) {
          if (a.det.kind == 1) {
            lsum += (double)ex * ex + (double)ey * ey + (double)ez * ez;
          } else {
            const int ax_ = a.det.axis;
            const float Eb = ax_ == 0 ? ey : (ax_ == 1 ? ez : ex);
            const float Ec2 = ax_ == 0 ? ez : (ax_ == 1 ? ex : ey);
            const float Hb2 = ax_ == 0 ? hy : (ax_ == 1 ? hz : hx);
            const float Hc2 = ax_ == 0 ? hz : (ax_ == 1 ? hx : hy);
            lsum += (double)Eb * Hc2 - (double)Ec2 * Hb2;
          }
        }
        q += g.plane;
      }
      c_hx = hx;
      c_hy = hy;
    }
    __syncthreads();
    if (tid == 0 && p + S <= R.p1) issue(p + S);
  }
  if (a.det.kind) {
    double v = lsum;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int wv = 0; wv < TY; ++wv) t += red[wv];
      if (t != 0.0) atomicAdd(a.obj, t);
    }
  }
}

// ======================================== reverse E phase (+ adjoint H) ===

template <int TY, int S>
__global__ void __launch_bounds__(32 * TY) k_lrev_e(const __grid_constant__ LagMaps m,
                                                   StepArgs a) {
  typedef G<TY> B;
  typedef LRE<TY, S> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
  const int x = x0 + tx, y = y0 + ty;
  const bool valid = x < g.nx && y < g.ny;
  const int k0 = blockIdx.z * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  const bool txs = tile_in_slab(x0, min(x0 + 32, g.nx - 1), g.nx, g.P);
  const bool tys = tile_in_slab(y0, min(y0 + TY, g.ny - 1), g.ny, g.P);
  const bool tint = x0 + 31 >= g.P && x0 < g.nx - g.P && y0 + TY - 1 >= g.P && y0 < g.ny - g.P;
  // plane k0-1: Ht(k0-1) at the own cell; planes k0..k1-1: the step proper;
  // plane p > k0 also finishes lam_H(p-1) with its +z neighbour terms.
  Ring<S> R = ring_setup<S>(dsm, Y::STAGE, k0 - 1, k1);
  // primal data only where the primal runs: interior tiles, planes P..nz-P-1
  // (and plane P-1's Ht for the z difference of plane P)
  auto primal_plane = [&](int p) { return tint && p >= g.P && p < g.nz - g.P; };
  auto issue = [&](int p) {
    unsigned char* st = R.at(p);
    uint64_t* bar = R.bar(p);
    const bool head = p < k0, body = p >= k0 && p < k1, tail = p > k0;
    const bool zs = p >= 0 && p < g.nz && in_slab(p, g.nz, g.P) && (body || tail);
    const bool lam = body || tail;
    const bool hbox = (head || body) && (primal_plane(p) || primal_plane(p + 1));
    const bool ebox = body && primal_plane(p);
    uint32_t bytes = (hbox ? 3 * B::P * 4 : 0) + (lam ? 4 * B::P * 4 : 0) +
                     (body ? 3 * B::OP * 4 : 0) + (ebox ? 3 * B::OP * 4 : 0) +
                     (body && txs ? 2 * B::XP * 4 : 0) + (body && tys ? 2 * B::YP * 4 : 0) +
                     (zs ? 2 * B::OP * 4 : 0);
    mbar_expect_tx(bar, bytes);
    if (hbox) tma_load_4d(st + Y::H, &m.Fw, bar, x0 - 4, y0 - 1, p, 3);
    if (lam) {
      tma_load_4d(st + Y::CB, &m.cbw, bar, x0, y0, p, 0);
      tma_load_4d(st + Y::LE, &m.Lw, bar, x0, y0, p, 0);
    }
    if (ebox) tma_load_4d(st + Y::E, &m.Fo, bar, x0, y0, p, 0);
    if (body) tma_load_4d(st + Y::LH, &m.Lo, bar, x0, y0, p, 3);
    if (body && txs) tma_load_4d(st + Y::PX, &m.Pxw, bar, x0, y0, p, 2);
    if (body && tys) tma_load_4d(st + Y::PY, &m.Pyw, bar, x0, y0, p, 6);
    if (zs) tma_load_4d(st + Y::PZ, &m.Po, bar, x0, y0, p, 10);
  };
  if (tid == 0)
    for (int p = R.p0; p <= R.p1 && p < R.p0 + S; ++p) issue(p);
  const bool sx = valid && in_slab(x, g.nx, g.P), sx1 = valid && x + 1 < g.nx && in_slab(x + 1, g.nx, g.P);
  const bool sy = valid && in_slab(y, g.ny, g.P), sy1 = valid && y + 1 < g.ny && in_slab(y + 1, g.ny, g.P);
  float bx = 0.f, ax = 0.f, kx = 1.f, bx1 = 0.f, ax1 = 0.f, kx1 = 1.f;
  float by = 0.f, ay = 0.f, ky = 1.f, by1 = 0.f, ay1 = 0.f, ky1 = 1.f;
  if (sx) { bx = prof(g, 0, PR_BE, x); ax = prof(g, 0, PR_AE, x); kx = prof(g, 0, PR_KE, x); }
  if (sx1) { bx1 = prof(g, 0, PR_BE, x + 1); ax1 = prof(g, 0, PR_AE, x + 1); kx1 = prof(g, 0, PR_KE, x + 1); }
  if (sy) { by = prof(g, 1, PR_BE, y); ay = prof(g, 1, PR_AE, y); ky = prof(g, 1, PR_KE, y); }
  if (sy1) { by1 = prof(g, 1, PR_BE, y + 1); ay1 = prof(g, 1, PR_AE, y + 1); ky1 = prof(g, 1, PR_KE, y + 1); }
  const bool xyin = x >= g.P && x < g.nx - g.P && y >= g.P && y < g.ny - g.P;
  const bool dxy = x >= a.dlo[0] && x < a.dhi[0] && y >= a.dlo[1] && y < a.dhi[1];
  const int dX = a.dhi[0] - a.dlo[0], dY = a.dhi[1] - a.dlo[1];
  const int lb = (ty + 1) * B::W + tx + 4;   // own cell in a lo box
  const int hb = ty * B::W + tx;             // own cell in a hi box
  const int ob = ty * 32 + tx;
  const long long nc = g.nc;
  float* F = a.F;
  float* LL = a.L;
  float* lpB = a.psiB;
  long long q = (long long)k0 * g.plane + (long long)y * g.px + x;
  float c_hx = 0.f, c_hy = 0.f;                                   // Ht(p-1) own
  float c_lhx = 0.f, c_lhy = 0.f, c_o8 = 0.f, c_o7 = 0.f, c_bx = 0.f, c_by = 0.f;  // lam_H(p-1)
  bool ok = true;
  for (int p = k0 - 1; p <= k1; ++p) {
    if (!R.wait(p)) ok = false;
    if (!__syncthreads_and(ok)) { ring_drain<S>(R, p, a.err); return; }
    const unsigned char* st = R.at(p);
    if (valid) {
      const float* CBb = reinterpret_cast<const float*>(st + Y::CB);
      const float* LEb = reinterpret_cast<const float*>(st + Y::LE);
      if (p > k0) {  // finish lam_H(p-1): the +z terms t7 (Ex,z,-) and t8 (Ey,z,+)
        const float c2 = CBb[hb];
        float n7 = -c2 * LEb[hb];
        float n8 = c2 * LEb[B::P + hb];
        if (p >= g.nz) { n7 = 0.f; n8 = 0.f; }
        if (p < g.nz && in_slab(p, g.nz, g.P)) {
          const float* P = reinterpret_cast<const float*>(st + Y::PZ);
          const float b1 = prof(g, 2, PR_BE, p), a1 = prof(g, 2, PR_AE, p), k1v = prof(g, 2, PR_KE, p);
          n7 = adj_s(n7, P[ob], lpB, 0, false, b1, a1, k1v);
          n8 = adj_s(n8, P[B::OP + ob], lpB, 0, false, b1, a1, k1v);
        }
        const long long qm = q - g.plane;
        LL[3 * nc + qm] = c_lhx + ((c_o8 - n8) + c_bx);
        LL[4 * nc + qm] = c_lhy + ((c_o7 - n7) + c_by);
      }
      if (p >= k0 && p < k1) {
        const int k = p;
        const float* Hb = reinterpret_cast<const float*>(st + Y::H);
        const float cbv = CBb[hb];
        const float lex = LEb[hb], ley = LEb[B::P + hb], lez = LEb[2 * B::P + hb];
        const bool hv = primal_plane(k) || primal_plane(k + 1);   // H box staged
        const float hx = hv ? Hb[lb] : 0.f, hy = hv ? Hb[B::P + lb] : 0.f;
        const float hz = hv ? Hb[2 * B::P + lb] : 0.f;
        // primal inverse E update on the interior, dL/dcb on the design box
        if (primal_plane(k) && xyin) {
          const float d6 = hz - Hb[2 * B::P + lb - B::W], d7 = hy - c_hy;
          const float d8 = hx - c_hx, d9 = hz - Hb[2 * B::P + lb - 1];
          const float d10 = hy - Hb[B::P + lb - 1], d11 = hx - Hb[lb - B::W];
          float c0 = d6 - d7, c1 = d8 - d9, c2 = d10 - d11;
          if (a.src.kind) {
            const float w = src_wt(a.src, x, y, k);
            if (w != 0.f) {
              const float wj = __fmul_rn(w, a.jn);
              if (a.src.comp == 0) c0 = __fsub_rn(c0, wj);
              else if (a.src.comp == 1) c1 = __fsub_rn(c1, wj);
              else c2 = __fsub_rn(c2, wj);
            }
          }
          const float* Eo = reinterpret_cast<const float*>(st + Y::E);
          F[q] = __fsub_rn(Eo[ob], __fmul_rn(cbv, c0));
          F[nc + q] = __fsub_rn(Eo[B::OP + ob], __fmul_rn(cbv, c1));
          F[2 * nc + q] = __fsub_rn(Eo[2 * B::OP + ob], __fmul_rn(cbv, c2));
          if (dxy && k >= a.dlo[2] && k < a.dhi[2]) {
            const float s = lex * c0 + ley * c1 + lez * c2;
            const long long qd = ((long long)(k - a.dlo[2]) * dY + (y - a.dlo[1])) * dX + (x - a.dlo[0]);
            a.gacc[qd] += (double)s;
          }
        }
        // adjoint of the E half-step, own and +x / +y terms
        const float wx = cbv * lex, wy = cbv * ley, wz = cbv * lez;
        float o6 = wx, o11 = -wz, o7 = -wx, o8 = wy, o9 = -wy, o10 = wz;
        float n6, n11, n9, n10;
        {
          const int r = hb + B::W;   // +y
          const float c2 = CBb[r];
          n6 = c2 * LEb[r];
          n11 = -c2 * LEb[2 * B::P + r];
        }
        {
          const int r = hb + 1;      // +x
          const float c2 = CBb[r];
          n9 = -c2 * LEb[B::P + r];
          n10 = c2 * LEb[2 * B::P + r];
        }
        if (y + 1 >= g.ny) { n6 = 0.f; n11 = 0.f; }
        if (x + 1 >= g.nx) { n9 = 0.f; n10 = 0.f; }
        if (sy || sy1) {
          const float* P = reinterpret_cast<const float*>(st + Y::PY);   // 32 x (TY+1) at (x0, y0)
          if (sy) {
            o6 = adj_s(o6, P[ob], lpB, 6 * nc + q, true, by, ay, ky);
            o11 = adj_s(o11, P[B::YP + ob], lpB, 7 * nc + q, true, by, ay, ky);
          }
          if (sy1) {
            n6 = adj_s(n6, P[ob + 32], lpB, 0, false, by1, ay1, ky1);
            n11 = adj_s(n11, P[B::YP + ob + 32], lpB, 0, false, by1, ay1, ky1);
          }
        }
        if (sx || sx1) {
          const float* P = reinterpret_cast<const float*>(st + Y::PX);   // 36 x TY at (x0, y0)
          const int xb = ty * 36 + tx;
          if (sx) {
            o9 = adj_s(o9, P[xb], lpB, 2 * nc + q, true, bx, ax, kx);
            o10 = adj_s(o10, P[B::XP + xb], lpB, 3 * nc + q, true, bx, ax, kx);
          }
          if (sx1) {
            n9 = adj_s(n9, P[xb + 1], lpB, 0, false, bx1, ax1, kx1);
            n10 = adj_s(n10, P[B::XP + xb + 1], lpB, 0, false, bx1, ax1, kx1);
          }
        }
        if (in_slab(k, g.nz, g.P)) {
          const float* P = reinterpret_cast<const float*>(st + Y::PZ);
          const float b = prof(g, 2, PR_BE, k), aa = prof(g, 2, PR_AE, k), kv = prof(g, 2, PR_KE, k);
          o7 = adj_s(o7, P[ob], lpB, 10 * nc + q, true, b, aa, kv);
          o8 = adj_s(o8, P[B::OP + ob], lpB, 11 * nc + q, true, b, aa, kv);
        }
        const float* LHo = reinterpret_cast<const float*>(st + Y::LH);
        LL[5 * nc + q] = LHo[2 * B::OP + ob] + ((o6 - n6) + (o9 - n9));
        c_lhx = LHo[ob];
        c_lhy = LHo[B::OP + ob];
        c_o8 = o8;
        c_o7 = o7;
        c_bx = o11 - n11;
        c_by = o10 - n10;
        c_hx = hx;
        c_hy = hy;
        q += g.plane;
      } else if (p < k0) {
        const float* Hb = reinterpret_cast<const float*>(st + Y::H);
        const bool hv = primal_plane(p) || primal_plane(p + 1);
        c_hx = hv ? Hb[lb] : 0.f;
        c_hy = hv ? Hb[B::P + lb] : 0.f;
      }
    }
    __syncthreads();
    if (tid == 0 && p + S <= R.p1) issue(p + S);
  }
}

// ======================================== reverse H phase (+ adjoint E) ===

template <int TY, int S>
__global__ void __launch_bounds__(32 * TY) k_lrev_h(const __grid_constant__ LagMaps m,
                                                   StepArgs a) {
  typedef G<TY> B;
  typedef LRH<TY, S> Y;
  extern __shared__ __align__(128) unsigned char dsm[];
  const Geo& g = a.g;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
  const int x = x0 + tx, y = y0 + ty;
  const bool valid = x < g.nx && y < g.ny;
  const int k0 = blockIdx.z * a.zchunk, k1 = min(g.nz, k0 + a.zchunk);
  const bool txs = tile_in_slab(max(x0 - 1, 0), min(x0 + 31, g.nx - 1), g.nx, g.P);
  const bool tys = tile_in_slab(max(y0 - 1, 0), min(y0 + TY - 1, g.ny - 1), g.ny, g.P);
  const bool tint = x0 + 31 >= g.P && x0 < g.nx - g.P && y0 + TY - 1 >= g.P && y0 < g.ny - g.P;
  // plane k0-1: lam_H(k0-1) terms for the -z neighbour; planes k0..k1-1: the
  // step proper; plane p > k0 also finishes the primal Ht(p-1) with E(p).
  Ring<S> R = ring_setup<S>(dsm, Y::STAGE, k0 - 1, k1);
  // primal data only where the primal runs: interior tiles, planes P..nz-P-1
  // (and plane nz-P's E for the z difference of plane nz-P-1)
  auto primal_plane = [&](int p) { return tint && p >= g.P && p < g.nz - g.P; };
  auto issue = [&](int p) {
    unsigned char* st = R.at(p);
    uint64_t* bar = R.bar(p);
    const bool head = p < k0, body = p >= k0 && p < k1, tail = p > k0;
    const bool zs = p >= 0 && p < g.nz && in_slab(p, g.nz, g.P) && (head || body);
    const bool ebox = (body && primal_plane(p)) || (tail && primal_plane(p - 1));
    const bool hown = body && primal_plane(p);
    uint32_t bytes = (ebox ? 3 * B::P * 4 : 0) + (head || body ? 3 * B::P * 4 : 0) +
                     (hown ? 3 * B::OP * 4 : 0) + (body ? 3 * B::OP * 4 : 0) +
                     (body && txs ? 2 * B::XP * 4 : 0) + (body && tys ? 2 * B::YP * 4 : 0) +
                     (zs ? 2 * B::OP * 4 : 0);
    mbar_expect_tx(bar, bytes);
    if (ebox) tma_load_4d(st + Y::E, &m.Fw, bar, x0, y0, p, 0);
    if (head || body) tma_load_4d(st + Y::LH, &m.Lw, bar, x0 - 4, y0 - 1, p, 3);
    if (hown) tma_load_4d(st + Y::H, &m.Fo, bar, x0, y0, p, 3);
    if (body) tma_load_4d(st + Y::LE, &m.Lo, bar, x0, y0, p, 0);
    if (body && txs) tma_load_4d(st + Y::PX, &m.Pxw, bar, x0 - 4, y0, p, 0);
    if (body && tys) tma_load_4d(st + Y::PY, &m.Pyw, bar, x0, y0 - 1, p, 4);
    if (zs) tma_load_4d(st + Y::PZ, &m.Po, bar, x0, y0, p, 8);
  };
  if (tid == 0)
    for (int p = R.p0; p <= R.p1 && p < R.p0 + S; ++p) issue(p);
  const bool sx = valid && in_slab(x, g.nx, g.P), sxm = valid && x > 0 && in_slab(x - 1, g.nx, g.P);
  const bool sy = valid && in_slab(y, g.ny, g.P), sym = valid && y > 0 && in_slab(y - 1, g.ny, g.P);
  float bx = 0.f, ax = 0.f, kx = 1.f, bxm = 0.f, axm = 0.f, kxm = 1.f;
  float by = 0.f, ay = 0.f, ky = 1.f, bym = 0.f, aym = 0.f, kym = 1.f;
  if (sx) { bx = prof(g, 0, PR_BH, x); ax = prof(g, 0, PR_AH, x); kx = prof(g, 0, PR_KH, x); }
  if (sxm) { bxm = prof(g, 0, PR_BH, x - 1); axm = prof(g, 0, PR_AH, x - 1); kxm = prof(g, 0, PR_KH, x - 1); }
  if (sy) { by = prof(g, 1, PR_BH, y); ay = prof(g, 1, PR_AH, y); ky = prof(g, 1, PR_KH, y); }
  if (sym) { bym = prof(g, 1, PR_BH, y - 1); aym = prof(g, 1, PR_AH, y - 1); kym = prof(g, 1, PR_KH, y - 1); }
  const bool xyin = x >= g.P && x < g.nx - g.P && y >= g.P && y < g.ny - g.P;
  const int lb = (ty + 1) * B::W + tx + 4;
  const int hb = ty * B::W + tx;
  const int ob = ty * 32 + tx;
  const float S_ = g.S;
  const long long nc = g.nc;
  float* F = a.F;
  float* LL = a.L;
  float* lpB = a.psiB;
  long long q = (long long)k0 * g.plane + (long long)y * g.px + x;
  float c_m1 = 0.f, c_m2 = 0.f;   // -z neighbour terms t1, t2 from plane p-1
  float c_d0 = 0.f, c_d3 = 0.f, c_d4 = 0.f, c_d5 = 0.f, c_ex = 0.f, c_ey = 0.f;
  float c_hx = 0.f, c_hy = 0.f, c_hz = 0.f;
  bool c_pr = false;              // primal Ht(p-1) pending
  bool ok = true;
  for (int p = k0 - 1; p <= k1; ++p) {
    if (!R.wait(p)) ok = false;
    if (!__syncthreads_and(ok)) { ring_drain<S>(R, p, a.err); return; }
    const unsigned char* st = R.at(p);
    if (valid) {
      const float* Eb = reinterpret_cast<const float*>(st + Y::E);
      if (p > k0 && c_pr) {  // finish the primal Ht(p-1) with dEy/dz, dEx/dz
        const float d1 = Eb[B::P + hb] - c_ey;
        const float d2 = Eb[hb] - c_ex;
        const long long qm = q - g.plane;
        F[3 * nc + qm] = __fadd_rn(c_hx, __fmul_rn(S_, c_d0 - d1));
        F[4 * nc + qm] = __fadd_rn(c_hy, __fmul_rn(S_, d2 - c_d3));
        F[5 * nc + qm] = __fadd_rn(c_hz, __fmul_rn(S_, c_d4 - c_d5));
      }
      const float* LHb = reinterpret_cast<const float*>(st + Y::LH);
      if (p >= k0 && p < k1) {
        const int k = p;
        c_pr = primal_plane(k) && xyin;
        if (c_pr) {  // primal Ht(k): x and y derivatives now, z derivatives next plane
          const float ex = Eb[hb], ey = Eb[B::P + hb], ez = Eb[2 * B::P + hb];
          const float* Ho = reinterpret_cast<const float*>(st + Y::H);
          c_d0 = Eb[2 * B::P + hb + B::W] - ez;
          c_d3 = Eb[2 * B::P + hb + 1] - ez;
          c_d4 = Eb[B::P + hb + 1] - ey;
          c_d5 = Eb[hb + B::W] - ex;
          c_ex = ex;
          c_ey = ey;
          c_hx = Ho[ob];
          c_hy = Ho[B::OP + ob];
          c_hz = Ho[2 * B::OP + ob];
        }
        // adjoint of the H half-step: lam_E += D^T lam_delta, v = -S s lam_H
        const float lhx = LHb[lb], lhy = LHb[B::P + lb], lhz = LHb[2 * B::P + lb];
        float o0 = -S_ * lhx, o5 = S_ * lhz, o1 = S_ * lhx, o2 = -S_ * lhy, o3 = S_ * lhy,
              o4 = -S_ * lhz;
        float m0 = -S_ * LHb[lb - B::W], m5 = S_ * LHb[2 * B::P + lb - B::W];   // -y
        float m3 = S_ * LHb[B::P + lb - 1], m4 = -S_ * LHb[2 * B::P + lb - 1];   // -x
        float m1 = c_m1, m2 = c_m2;                                              // -z
        if (y == 0) { m0 = 0.f; m5 = 0.f; }
        if (x == 0) { m3 = 0.f; m4 = 0.f; }
        if (sy || sym) {
          const float* P = reinterpret_cast<const float*>(st + Y::PY);   // 32 x (TY+1) at (x0, y0-1)
          const int yb = (ty + 1) * 32 + tx;
          if (sy) {
            o0 = adj_s(o0, P[yb], lpB, 4 * nc + q, true, by, ay, ky);
            o5 = adj_s(o5, P[B::YP + yb], lpB, 5 * nc + q, true, by, ay, ky);
          }
          if (sym) {
            m0 = adj_s(m0, P[yb - 32], lpB, 0, false, bym, aym, kym);
            m5 = adj_s(m5, P[B::YP + yb - 32], lpB, 0, false, bym, aym, kym);
          }
        }
        if (sx || sxm) {
          const float* P = reinterpret_cast<const float*>(st + Y::PX);   // 36 x TY at (x0-4, y0)
          const int xb = ty * 36 + tx + 4;
          if (sx) {
            o3 = adj_s(o3, P[xb], lpB, 0 * nc + q, true, bx, ax, kx);
            o4 = adj_s(o4, P[B::XP + xb], lpB, 1 * nc + q, true, bx, ax, kx);
          }
          if (sxm) {
            m3 = adj_s(m3, P[xb - 1], lpB, 0, false, bxm, axm, kxm);
            m4 = adj_s(m4, P[B::XP + xb - 1], lpB, 0, false, bxm, axm, kxm);
          }
        }
        const bool sz = in_slab(k, g.nz, g.P);
        if (sz) {
          const float* P = reinterpret_cast<const float*>(st + Y::PZ);
          const float b = prof(g, 2, PR_BH, k), aa = prof(g, 2, PR_AH, k), kv = prof(g, 2, PR_KH, k);
          o1 = adj_s(o1, P[ob], lpB, 8 * nc + q, true, b, aa, kv);
          o2 = adj_s(o2, P[B::OP + ob], lpB, 9 * nc + q, true, b, aa, kv);
        }
        const float* LEo = reinterpret_cast<const float*>(st + Y::LE);
        LL[q] = LEo[ob] + ((m2 - o2) + (m5 - o5));
        LL[nc + q] = LEo[B::OP + ob] + ((m1 - o1) + (m4 - o4));
        LL[2 * nc + q] = LEo[2 * B::OP + ob] + ((m0 - o0) + (m3 - o3));
        q += g.plane;
      }
      if (p < k1) {  // -z neighbour terms for plane p+1: t1 (Hx,z,-), t2 (Hy,z,+) at plane p
        float m1n = S_ * LHb[lb], m2n = -S_ * LHb[B::P + lb];
        if (p >= 0 && in_slab(p, g.nz, g.P)) {
          const float* P = reinterpret_cast<const float*>(st + Y::PZ);
          const float b1 = prof(g, 2, PR_BH, p), a1 = prof(g, 2, PR_AH, p), k1v = prof(g, 2, PR_KH, p);
          m1n = adj_s(m1n, P[ob], lpB, 0, false, b1, a1, k1v);
          m2n = adj_s(m2n, P[B::OP + ob], lpB, 0, false, b1, a1, k1v);
        }
        c_m1 = p >= 0 ? m1n : 0.f;
        c_m2 = p >= 0 ? m2n : 0.f;
      }
    }
    __syncthreads();
    if (tid == 0 && p + S <= R.p1) issue(p + S);
  }
}

// ------------------------------------------------------------ launchers ---
template <class KT>
static cudaError_t set_smem_l(KT kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int TY, int S>
static cudaError_t launch_lag_t(int which, const LagMaps& m, const StepArgs& a, cudaStream_t s) {
  dim3 grid((a.g.nx + 31) / 32, (a.g.ny + TY - 1) / TY, (a.g.nz + a.zchunk - 1) / a.zchunk);
  dim3 block(32, TY);
  cudaError_t e = cudaSuccess;
  switch (which) {
    case 0: {
      int sm = LFH<TY, S>::smem();
      if ((e = set_smem_l(k_lfwd_h<TY, S>, sm))) return e;
      k_lfwd_h<TY, S><<<grid, block, sm, s>>>(m, a);
      break;
    }
    case 1: {
      int sm = LFE<TY, S>::smem();
      if ((e = set_smem_l(k_lfwd_e<TY, S>, sm))) return e;
      k_lfwd_e<TY, S><<<grid, block, sm, s>>>(m, a);
      break;
    }
    case 2: {
      int sm = LRE<TY, S>::smem();
      if ((e = set_smem_l(k_lrev_e<TY, S>, sm))) return e;
      k_lrev_e<TY, S><<<grid, block, sm, s>>>(m, a);
      break;
    }
    case 3: {
      int sm = LRH<TY, S>::smem();
      if ((e = set_smem_l(k_lrev_h<TY, S>, sm))) return e;
      k_lrev_h<TY, S><<<grid, block, sm, s>>>(m, a);
      break;
    }
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// which: 0 forward H, 1 forward E, 2 reverse E phase, 3 reverse H phase.
// Stage counts 2 and 4 are built for tile heights 2, 4 and 8; the other
// heights run with 3.
cudaError_t launch_lag(int which, const LagMaps& m, const StepArgs& a, cudaStream_t s) {
  const int S = a.stages;
  switch (a.tile_y) {
    case 1: return launch_lag_t<1, 3>(which, m, a, s);
    case 2: return S == 2 ? launch_lag_t<2, 2>(which, m, a, s)
                 : S == 4 ? launch_lag_t<2, 4>(which, m, a, s) : launch_lag_t<2, 3>(which, m, a, s);
    case 4: return S == 2 ? launch_lag_t<4, 2>(which, m, a, s)
                 : S == 4 ? launch_lag_t<4, 4>(which, m, a, s) : launch_lag_t<4, 3>(which, m, a, s);
    case 8: return S == 2 ? launch_lag_t<8, 2>(which, m, a, s)
                 : S == 4 ? launch_lag_t<8, 4>(which, m, a, s) : launch_lag_t<8, 3>(which, m, a, s);
    case 16: return launch_lag_t<16, 3>(which, m, a, s);
  }
  return cudaErrorInvalidValue;
}

// -------------------------------------------------------- tensor maps ---
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn3() {
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

static cudaError_t enc3(CUtensorMap* m, const float* base, const Geo& g, int ncomp, int bx, int by,
                        int bc) {
  auto fn = encode_fn3();
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

// 4D view (x, y, z, component) of one axis array of an auxiliary set.
static cudaError_t enc_axis(CUtensorMap* m, const float* set, const PsiAxis& A, int bx, int by) {
  auto fn = encode_fn3();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[4] = {(cuuint64_t)A.e0, (cuuint64_t)A.d1, (cuuint64_t)A.d2, 4};
  cuuint64_t strides[3] = {(cuuint64_t)A.d0 * 4, (cuuint64_t)A.d0 * A.d1 * 4,
                           (cuuint64_t)A.cs * 4};
  cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 2};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(set + A.off), dims,
                  strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t encode_lag_maps(const float* F, const float* Lm, const float* cb, const float* psiA,
                            const Geo& g, int ty, int tw, const PsiLayout& pl, LagMaps* m) {
  *m = LagMaps{};
  cudaError_t e;
  const int w = tw + 4;
  if ((e = enc_axis(&m->Qxo, psiA, pl.ax[0], tw, ty))) return e;
  if ((e = enc_axis(&m->Qxw, psiA, pl.ax[0], w, ty))) return e;
  if ((e = enc_axis(&m->Qyo, psiA, pl.ax[1], tw, ty))) return e;
  if ((e = enc_axis(&m->Qyw, psiA, pl.ax[1], tw, ty + 1))) return e;
  if ((e = enc_axis(&m->Qzo, psiA, pl.ax[2], tw, ty))) return e;
  if ((e = enc3(&m->Fw, F, g, 6, w, ty + 1, 3))) return e;
  if ((e = enc3(&m->Fo, F, g, 6, tw, ty, 3))) return e;
  if ((e = enc3(&m->Lw, Lm, g, 6, w, ty + 1, 3))) return e;
  if ((e = enc3(&m->Lo, Lm, g, 6, tw, ty, 3))) return e;
  if ((e = enc3(&m->cbw, cb, g, 1, w, ty + 1, 1))) return e;
  if ((e = enc3(&m->cbo, cb, g, 1, tw, ty, 1))) return e;
  // the one-cell kernels stage the full-grid set as 12 components
  if (pl.total != 12 * g.nc) return cudaSuccess;
  if ((e = enc3(&m->Pxw, psiA, g, 12, w, ty, 2))) return e;
  if ((e = enc3(&m->Pyw, psiA, g, 12, tw, ty + 1, 2))) return e;
  return enc3(&m->Po, psiA, g, 12, tw, ty, 2);
}

}  // namespace fdtd
