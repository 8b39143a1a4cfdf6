// kernels_fused.cu -- fused 2.5D forward / reverse step kernels (in progress).
#include "fdtd_internal.cuh"

namespace fdtd {

cudaError_t launch_fused_fwd(const StepArgs&, float*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_fused_rev(const StepArgs&, float*, float*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace fdtd
