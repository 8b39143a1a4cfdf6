// restore_fused.cuh -- the reverse step's tape restore and objective seeding
// carried by the reverse-phase launches of the two-cells-per-thread kernels
// instead of a launch of their own.
//
// Reverse step n needs (Sec. 2), before its E phase: Ht^{n+1/2} on the low
// interface layers and the seeds dl_n/d(E^{n+1}) on lam_E; before its H
// phase: E^n on the high layers; and the seeds dl_n/d(Ht^{n+1/2}) on lam_H
// before the E phase reads lam_H.  None of these values is read by the launch
// that carries it:
//   * the H phase of step n+1 restores Ht^{n+1/2} on the low layers (it
//     neither reads nor writes Ht outside the interior) and adds the lam_E
//     seeds of step n to the lam_E it writes (it is the only reader and writer
//     of a cell's lam_E, and it has E^{n+1} and, one plane later, the
//     Ht^{n+1/2} it computes);
//   * the E phase of step n restores E^n on the high layers (it reads E only
//     inside the interior) and adds the lam_H seeds of step n to the lam_H it
//     loads for its own cells (lam_H is read without a halo there).
// CTAs past the tile grid (grid z beyond the z chunks) do the face restores;
// the tile CTAs add the seeds of their own cells.
#pragma once

#include "bdct.cuh"
#include "tape_common.cuh"

namespace fdtd {

struct FusedRestore {
  int faces;               // 0: none; 1: Ht on the low faces; 2: E on the high faces
  int seed;                // 0: none; 1: lam_E seeds (H phase); 2: lam_H seeds (E phase)
  int dtype;               // tape type (0..9)
  int extra_z;             // grid z planes of face-restoring CTAs past the z chunks
  const unsigned char* tape;
  long long stride;        // bytes per tape sample
  const float* scales;     // per-face, per-sample scales [J][6]
  const float* beta;       // BDCT basis [64 coefficients][64 cells]
  Interp ip;               // slots and weights of the restored step
  Faces fc;
  BdctLayout bl;
  Det det, det2;
  const double* seeds;     // device FP64 seeds of det and det2
};

// Recorded value rr of face f in tape sample s (decoded, times its scale).
__device__ __forceinline__ float fr_decode(const FusedRestore& R, int s, int f, int rr) {
  const unsigned char* smp = R.tape + (long long)s * R.stride;
  const FaceDesc& fd = R.fc.f[f];
  const long long i = fd.off + rr;
  float x = 0.f;
  switch (R.dtype) {
    case 0: return reinterpret_cast<const float*>(smp)[i];
    case 1: return Code<1>::dec(reinterpret_cast<const Code<1>::T*>(smp)[i]);
    case 2: x = Code<2>::dec(reinterpret_cast<const Code<2>::T*>(smp)[i]); break;
    case 3: x = Code<3>::dec(reinterpret_cast<const Code<3>::T*>(smp)[i]); break;
    case 4: x = Code<4>::dec(reinterpret_cast<const Code<4>::T*>(smp)[i]); break;
    case 5: x = Code<5>::dec(reinterpret_cast<const Code<5>::T*>(smp)[i]); break;
    case 6: x = Code<6>::dec(reinterpret_cast<const Code<6>::T*>(smp)[i]); break;
    case 7: x = Code<7>::dec(reinterpret_cast<const Code<7>::T*>(smp)[i]); break;
    case 8: x = Code<8>::dec(reinterpret_cast<const Code<8>::T*>(smp)[i]); break;
    default: {   // block-transform codec
      const int row = rr / fd.nu, u = rr - row * fd.nu;
      const int comp_t = row >= fd.nv, v = row - comp_t * fd.nv;
      const int b = R.bl.bstart[f] + comp_t * R.bl.nbu[f] * R.bl.nbv[f] + (v >> 3) * R.bl.nbu[f] +
                    (u >> 3);
      const int t = (v & 7) * 8 + (u & 7);
      const signed char* codes = reinterpret_cast<const signed char*>(smp) + (long long)b * R.bl.K;
      float acc = 0.f;
      for (int c = 0; c < R.bl.K; ++c)
        acc = __fmaf_rn((float)codes[c], __ldg(R.beta + c * 64 + t), acc);
      return __fmul_rn(acc, __ldg(reinterpret_cast<const float*>(smp + R.bl.code_bytes) + b));
    }
  }
  return x * __ldg(R.scales + s * 6 + f);
}

// Face restore by extra CTA bid of nb: the three faces of one field (low
// faces f = 0, 2, 4 for Ht; high faces 1, 3, 5 for E), the value at this
// reverse step being sum_m w[m] * sample(slot[m]), as the restore launch.
__device__ __forceinline__ void fr_faces(const FusedRestore& R, const Geo& g, float* __restrict__ F,
                                         int bid, int nb) {
  const int fld = R.faces - 1;
  const int n0 = R.fc.start[fld + 1] - R.fc.start[fld];
  const int n1 = R.fc.start[fld + 3] - R.fc.start[fld + 2];
  const int n2 = R.fc.start[fld + 5] - R.fc.start[fld + 4];
  const int total = n0 + n1 + n2;
  const int nthr = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int r = bid * nthr + tid; r < total; r += nb * nthr) {
    const int f = r < n0 ? fld : (r < n0 + n1 ? fld + 2 : fld + 4);
    const int rr = r < n0 ? r : (r < n0 + n1 ? r - n0 : r - n0 - n1);
    float val = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int s = R.ip.slot[fld][m];
      if (s >= 0) val += R.ip.w[fld][m] * fr_decode(R, s, f, rr);
    }
    int comp;
    const long long q = face_value_cell(g, R.fc.f[f], rr, &comp);
    F[comp * g.nc + q] = val;
  }
}

// Is cell (i, j, k) on the detector plane?
__device__ __forceinline__ bool det_hit(const Det& d, int i, int j, int k) {
  if (!d.kind) return false;
  int u, v;
  return on_plane(d.axis, d.index, d.u0, d.u1, d.v0, d.v1, i, j, k, &u, &v);
}

}  // namespace fdtd
