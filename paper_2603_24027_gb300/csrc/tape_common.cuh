// tape_common.cuh -- addressing shared by the tape kernels: the cells of the
// recorded faces and the detector seeding of the reverse step.
#pragma once

#include "fdtd_internal.cuh"

namespace fdtd {

// Cell at (u, v) of the plane normal to `axis` at `index`; (u, v) are the
// two other axes in increasing order.
__device__ __forceinline__ long long cell_on_plane(const Geo& g, int axis, int index, int u,
                                                   int v) {
  const int x = axis == 0 ? index : u;
  const int y = axis == 1 ? index : (axis == 0 ? u : v);
  const int z = axis == 2 ? index : v;
  return (long long)z * g.plane + (long long)y * g.px + x;
}

// Value r of face fd ([comp][v][u]): its field component and cell.
__device__ __forceinline__ long long face_value_cell(const Geo& g, const FaceDesc& fd, int r,
                                                    int* comp) {
  const int row = r / fd.nu, u = r - row * fd.nu;
  const int t = row >= fd.nv, v = row - t * fd.nv;
  *comp = t ? fd.comp1 : fd.comp0;
  return cell_on_plane(g, fd.axis, fd.layer, g.P + u, g.P + v);
}

// Detector blocks of the restore launch: block b (of det_blocks per
// detector) adds the objective seeds on the detector planes: seeds[0] *
// dl_n/d(E^{n+1}, Ht^{n+1/2}) for the detector, seeds[1] * dm_n/d(...) for the
// second one (E2_PLANE: 2 s E; POYNTING_PLANE: the cross-product terms).
__device__ __forceinline__ void seed_detectors(float* __restrict__ F, float* __restrict__ L,
                                               const Geo& g, const Det& det, const Det& det2,
                                               const double* __restrict__ seeds, int b,
                                               int det_blocks) {
  const int which = b >= det_blocks;
  const Det& d = which ? det2 : det;
  if (!d.kind) return;
  const int du = d.u1 - d.u0, dv = d.v1 - d.v0;
  const int r = (b - which * det_blocks) * blockDim.x + threadIdx.x;
  if (r >= du * dv) return;
  const float s = (float)seeds[which];
  const int v = r / du, e = r - v * du;
  const long long q = cell_on_plane(g, d.axis, d.index, d.u0 + e, d.v0 + v);
  if (d.kind == 1) {
    for (int c = 0; c < 3; ++c) L[c * g.nc + q] += s * (2.0f * F[c * g.nc + q]);
  } else {
    const int bb = (d.axis + 1) % 3, c = (d.axis + 2) % 3;
    const float Eb = F[bb * g.nc + q], Ec = F[c * g.nc + q];
    const float Hb = F[(3 + bb) * g.nc + q], Hc = F[(3 + c) * g.nc + q];
    L[bb * g.nc + q] += s * Hc;
    L[c * g.nc + q] -= s * Hb;
    L[(3 + c) * g.nc + q] += s * Eb;
    L[(3 + bb) * g.nc + q] -= s * Ec;
  }
}

}  // namespace fdtd
