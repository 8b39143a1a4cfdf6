// tensor_maps.cu -- TMA tensor maps of the plane-staging kernels.
//
// Every field array is viewed as a 4D tensor (x, y, z, component) of float32
// with the padded row pitch, so one box load stages a tile of several
// components of one z plane.  Out-of-range box elements arrive as zeros: the
// zero-padding boundary of the grid.  The CPML auxiliary arrays are viewed per
// axis (x, y, z-or-slab-row, 4 components).
#include <cudaTypedefs.h>

#include "fdtd_internal.cuh"

namespace fdtd {

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
                            const Geo& g, int ty, int tw, const PsiLayout& pl, LagMaps* m,
                            const float* Fwide) {
  *m = LagMaps{};
  cudaError_t e;
  const int w = tw + 4;
  if ((e = enc_axis(&m->Qxo, psiA, pl.ax[0], tw, ty))) return e;
  if ((e = enc_axis(&m->Qxw, psiA, pl.ax[0], w, ty))) return e;
  if ((e = enc_axis(&m->Qyo, psiA, pl.ax[1], tw, ty))) return e;
  if ((e = enc_axis(&m->Qyw, psiA, pl.ax[1], tw, ty + 1))) return e;
  if ((e = enc_axis(&m->Qzo, psiA, pl.ax[2], tw, ty))) return e;
  if ((e = enc3(&m->Fw, Fwide ? Fwide : F, g, 6, w, ty + 1, 3))) return e;
  if ((e = enc3(&m->Fo, F, g, 6, tw, ty, 3))) return e;
  if ((e = enc3(&m->Lw, Lm, g, 6, w, ty + 1, 3))) return e;
  if ((e = enc3(&m->Lo, Lm, g, 6, tw, ty, 3))) return e;
  if ((e = enc3(&m->cbw, cb, g, 1, w, ty + 1, 1))) return e;
  if ((e = enc3(&m->cbo, cb, g, 1, tw, ty, 1))) return e;
  return cudaSuccess;
}

cudaError_t encode_rev_maps(const float* F, const float* Lm, const float* cb, const float* psiA,
                            const Geo& g, const PsiLayout& pl, RevMaps* m) {
  const int tw = 32, ty = 8;
  *m = RevMaps{};
  cudaError_t e;
  if ((e = enc3(&m->F40, F, g, 6, tw + 8, ty + 2, 3))) return e;
  if ((e = enc3(&m->F36, F, g, 6, tw + 4, ty + 1, 3))) return e;
  if ((e = enc3(&m->cb36, cb, g, 1, tw + 4, ty + 1, 1))) return e;
  if ((e = enc3(&m->cb40, cb, g, 1, tw + 8, ty + 2, 1))) return e;
  if ((e = enc3(&m->cb32, cb, g, 1, tw, ty, 1))) return e;
  if ((e = enc3(&m->L40, Lm, g, 6, tw + 8, ty + 2, 3))) return e;
  if ((e = enc3(&m->L36, Lm, g, 6, tw + 4, ty + 1, 3))) return e;
  if ((e = enc_axis(&m->Qx40, psiA, pl.ax[0], tw + 8, ty + 1))) return e;
  if ((e = enc_axis(&m->Qy36, psiA, pl.ax[1], tw + 4, ty + 2))) return e;
  if ((e = enc_axis(&m->Qz36, psiA, pl.ax[2], tw + 4, ty + 1))) return e;
  if ((e = enc_axis(&m->Qxw, psiA, pl.ax[0], tw + 4, ty))) return e;
  if ((e = enc_axis(&m->Qyw, psiA, pl.ax[1], tw, ty + 1))) return e;
  return enc_axis(&m->Qzo, psiA, pl.ax[2], tw, ty);
}

cudaError_t encode_fwd2_maps(const float* F, const float* cb, const Geo& g, Fwd2Maps* m) {
  *m = Fwd2Maps{};
  cudaError_t e;
  if ((e = enc3(&m->F4012, F, g, 6, 40, 12, 3))) return e;
  return enc3(&m->cb40, cb, g, 1, 40, 10, 1);
}

}  // namespace fdtd
