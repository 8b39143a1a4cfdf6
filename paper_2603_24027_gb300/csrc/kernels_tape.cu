// kernels_tape.cu -- boundary tape: record (compress) and restore (decompress).
//
// Sec. 2: the fields on the interface slices between the simulation volume
// and the PML are recorded in the forward run and injected back in the
// time-reversed run; they are stored at reduced bit-width (converted back to
// FP32 before use) and only every k-th step, with interpolation in time.
//
// Recorded layers (the values the interior inverse reads from outside the
// interior): low faces (x-, y-, z-) at index P-1 hold the two tangential Ht
// components at n+1/2; high faces (x+, y+, z+) at index N-P hold the two
// tangential E components at n.  One sample = 6 faces x 2 components x the
// interior cross-section, [face][comp][v][u].
//
// Scaled formats: k_record runs one thread-block cluster per face: every CTA
// takes a share of the face, the per-face absmax is reduced across the
// cluster through distributed shared memory, then each CTA encodes its share
// with the common scale (no global atomics, no second launch).  Unscaled
// formats use one thread per value.
#include <cooperative_groups.h>

#include <type_traits>

#include "tape_common.cuh"

namespace cg = cooperative_groups;

namespace fdtd {

// Call fn(std::integral_constant<int, DT>) for the tape element type dtype.
template <class Fn>
static cudaError_t with_dtype(int dtype, Fn&& fn) {
  switch (dtype) {
    case 0: return fn(std::integral_constant<int, 0>{});
    case 1: return fn(std::integral_constant<int, 1>{});
    case 2: return fn(std::integral_constant<int, 2>{});
    case 3: return fn(std::integral_constant<int, 3>{});
    case 4: return fn(std::integral_constant<int, 4>{});
    case 5: return fn(std::integral_constant<int, 5>{});
    case 6: return fn(std::integral_constant<int, 6>{});
    case 7: return fn(std::integral_constant<int, 7>{});
    case 8: return fn(std::integral_constant<int, 8>{});
  }
  return cudaErrorInvalidValue;
}

// Smallest per-face scale: the smallest normal FP32 number, so that
// amax / format_max never underflows to zero (0/0 would encode NaN).
static constexpr float kMinScale = 1.17549435e-38f;

static constexpr int REC_CLUSTER = 8;     // raw codec entry points
static constexpr int REC_THREADS = 512;
static constexpr int FACE_CLUSTER = 16;   // CTAs per face when a face-wide absmax is needed
static constexpr int FACE_THREADS = 1024;
static constexpr int FLAT_THREADS = 256;  // one thread per value otherwise

// Unscaled formats: one thread per recorded value, grid (value blocks, face).
template <int DT>
__device__ __forceinline__ void record_flat_body(const float* __restrict__ FH,
                                                 const float* __restrict__ FE, const Geo& g,
                                                 const Faces& fc, void* __restrict__ tape_sample,
                                                 float* scale_slot) {
  typedef typename Code<DT>::T T;
  const int f = blockIdx.y;
  const FaceDesc& fd = fc.f[f];
  const int n = 2 * fd.nu * fd.nv;
  const int r = blockIdx.x * FLAT_THREADS + threadIdx.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) scale_slot[f] = 1.0f;
  if (r >= n) return;
  const float* __restrict__ F = (f & 1) ? FE : FH;
  int comp;
  const long long q = face_value_cell(g, fd, r, &comp);
  reinterpret_cast<T*>(tape_sample)[fd.off + r] = Code<DT>::enc(F[comp * g.nc + q]);
}

template <int DT>
__global__ void __launch_bounds__(FLAT_THREADS) k_record_flat(const float* __restrict__ FH,
                                                              const float* __restrict__ FE, Geo g,
                                                              const __grid_constant__ Faces fc,
                                                              void* __restrict__ tape_sample,
                                                              float* scale_slot) {
  record_flat_body<DT>(FH, FE, g, fc, tape_sample, scale_slot);
}

// Batched designs: the same for the job blockIdx.z of a list.
template <int DT>
__global__ void __launch_bounds__(FLAT_THREADS) k_record_flat_batch(const RecordJob* __restrict__ jobs) {
  const RecordJob& j = jobs[blockIdx.z];
  record_flat_body<DT>(j.FH, j.FE, j.g, j.fc, j.sample, j.scale_slot);
}

// Scaled formats: one cluster of FACE_CLUSTER CTAs per face (blockIdx.y); the
// face's absmax is reduced across the cluster through distributed shared
// memory, then each CTA encodes its share with the common scale.
template <int DT>
__global__ void __launch_bounds__(FACE_THREADS) k_record(const float* __restrict__ FH,
                                                         const float* __restrict__ FE, Geo g,
                                                         const __grid_constant__ Faces fc,
                                                         void* __restrict__ tape_sample,
                                                         float* scale_slot) {
  typedef typename Code<DT>::T T;
  __shared__ float red[FACE_THREADS / 32];
  __shared__ float cl_amax;
  cg::cluster_group cluster = cg::this_cluster();
  const int f = blockIdx.y;
  const FaceDesc& fd = fc.f[f];
  const float* __restrict__ F = (f & 1) ? FE : FH;
  const int n = 2 * fd.nu * fd.nv;
  const int rank = (int)cluster.block_rank();
  const int nr = (int)cluster.num_blocks();
  const int tid = threadIdx.x;
  float m = 0.f;
  for (int r = rank * FACE_THREADS + tid; r < n; r += nr * FACE_THREADS) {
    int comp;
    const long long q = face_value_cell(g, fd, r, &comp);
    m = fmaxf(m, fabsf(F[comp * g.nc + q]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  if (tid < 32) {
    float t = red[tid];
    for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (tid == 0) cl_amax = t;
  }
  cluster.sync();
  float amax = 0.f;
  for (int b = 0; b < nr; ++b) amax = fmaxf(amax, *cluster.map_shared_rank(&cl_amax, b));
  cluster.sync();  // peers may still be reading this CTA's cl_amax
  const float scale = amax > 0.f ? fmaxf(__fdiv_rn(amax, Code<DT>::fmax), kMinScale) : 1.0f;
  if (rank == 0 && tid == 0) scale_slot[f] = scale;
  T* out = reinterpret_cast<T*>(tape_sample) + fd.off;
  for (int r = rank * FACE_THREADS + tid; r < n; r += nr * FACE_THREADS) {
    int comp;
    const long long q = face_value_cell(g, fd, r, &comp);
    out[r] = Code<DT>::enc(__fdiv_rn(F[comp * g.nc + q], scale));
  }
}

template <int DT>
static cudaError_t launch_record_t(int scaled, const float* FH, const float* FE, Geo g,
                                   const Faces& fc, void* tape_sample, float* scale_slot,
                                   cudaStream_t s) {
  if (!scaled) {
    int nmax = 0;
    for (int f = 0; f < 6; ++f) nmax = max(nmax, 2 * fc.f[f].nu * fc.f[f].nv);
    dim3 grid((nmax + FLAT_THREADS - 1) / FLAT_THREADS, 6);
    k_record_flat<DT><<<grid, FLAT_THREADS, 0, s>>>(FH, FE, g, fc, tape_sample, scale_slot);
    return cudaGetLastError();
  }
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_record<DT>,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e) return e;
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(FACE_CLUSTER, 6, 1);
  cfg.blockDim = dim3(FACE_THREADS, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attrs[1];
  attrs[0].id = cudaLaunchAttributeClusterDimension;
  attrs[0].val.clusterDim.x = FACE_CLUSTER;
  attrs[0].val.clusterDim.y = 1;
  attrs[0].val.clusterDim.z = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_record<DT>, FH, FE, g, fc, tape_sample, scale_slot);
}

cudaError_t launch_record(int dtype, int scaled, const float* FH, const float* FE, Geo g,
                          const Faces& fc, void* tape_sample, float* scale_slot, cudaStream_t s) {
  // FP32 and BF16 are never scaled
  return with_dtype(dtype, [&](auto dt) {
    constexpr int DT = decltype(dt)::value;
    return launch_record_t<DT>(DT >= 2 ? scaled : 0, FH, FE, g, fc, tape_sample, scale_slot, s);
  });
}

// -------------------------------------------------------------- restore ---
// One thread per recorded value over all six faces (value r of the sample
// belongs to the face f with start[f] <= r < start[f+1]): the value at this
// reverse step is sum_m w[m] * decode(sample slot[m]) * scale[slot[m]] (slot
// -1 = the known zero initial state or an unused term).  The blocks after the
// faces' add the objective seeds on the detector planes: seeds[0] *
// dl_n/d(E^{n+1}, Ht^{n+1/2}) for the detector, seeds[1] * dm_n/d(...) for
// the second one.
template <int DT>
__device__ __forceinline__ void restore_seed_body(float* __restrict__ F, float* __restrict__ L,
                                                  const Geo& g, const Faces& fc,
                                                  const void* __restrict__ tape, long long stride,
                                                  const float* __restrict__ scales,
                                                  const Interp& ip, const Det& det,
                                                  const Det& det2,
                                                  const double* __restrict__ seeds,
                                                  int face_blocks, int det_blocks) {
  typedef typename Code<DT>::T T;
  if ((int)blockIdx.x < face_blocks) {
    const int r = blockIdx.x * FLAT_THREADS + threadIdx.x;
    if (r >= fc.start[6]) return;
    int f = 0;
#pragma unroll
    for (int t = 1; t < 6; ++t) f += r >= fc.start[t];
    const FaceDesc& fd = fc.f[f];
    const int rr = r - fc.start[f];
    const int fld = f & 1;  // 0: Ht on low faces, 1: E on high faces
    const T* tp = reinterpret_cast<const T*>(tape) + fd.off + rr;
    float val = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int s = ip.slot[fld][m];
      if (s >= 0) {
        float x = Code<DT>::dec(tp[(long long)s * stride]);
        if (DT >= 2) x = x * __ldg(scales + s * 6 + f);
        val += ip.w[fld][m] * x;
      }
    }
    int comp;
    const long long q = face_value_cell(g, fd, rr, &comp);
    F[comp * g.nc + q] = val;
    return;
  }
  seed_detectors(F, L, g, det, det2, seeds, blockIdx.x - face_blocks, det_blocks);
}

template <int DT>
__global__ void __launch_bounds__(FLAT_THREADS) k_restore_seed(float* __restrict__ F,
                                                               float* __restrict__ L, Geo g,
                                                               const __grid_constant__ Faces fc,
                                                               const void* __restrict__ tape,
                                                               long long stride,
                                                               const float* __restrict__ scales,
                                                               const __grid_constant__ Interp ip,
                                                               Det det, Det det2,
                                                               const double* __restrict__ seeds,
                                                               int face_blocks, int det_blocks) {
  restore_seed_body<DT>(F, L, g, fc, tape, stride, scales, ip, det, det2, seeds, face_blocks,
                        det_blocks);
}

// Batched designs: the same for the job blockIdx.y of a list (blocks past the
// job's own face and detector blocks return).
template <int DT>
__global__ void __launch_bounds__(FLAT_THREADS) k_restore_seed_batch(const RestoreJob* __restrict__ jobs) {
  const RestoreJob& j = jobs[blockIdx.y];
  if ((int)blockIdx.x >= j.face_blocks + (j.det2.kind ? 2 : 1) * j.det_blocks) return;
  restore_seed_body<DT>(j.F, j.L, j.g, j.fc, j.tape, j.stride, j.scales, j.ip, j.det, j.det2,
                        j.seeds, j.face_blocks, j.det_blocks);
}

cudaError_t launch_restore_seed(int dtype, float* F, float* L, Geo g, const Faces& fc,
                                const void* tape, long long stride, const float* scales,
                                const Interp& ip, const Det& det, const Det& det2,
                                const double* seeds, cudaStream_t s) {
  const int face_blocks = (fc.start[6] + FLAT_THREADS - 1) / FLAT_THREADS;
  int dmax = det.kind ? (det.u1 - det.u0) * (det.v1 - det.v0) : 0;
  if (det2.kind) dmax = max(dmax, (det2.u1 - det2.u0) * (det2.v1 - det2.v0));
  const int det_blocks = (dmax + FLAT_THREADS - 1) / FLAT_THREADS;
  const int blocks = face_blocks + (det2.kind ? 2 : 1) * det_blocks;
  if (blocks == 0) return cudaSuccess;
  return with_dtype(dtype, [&](auto dt) {
    constexpr int DT = decltype(dt)::value;
    k_restore_seed<DT><<<blocks, FLAT_THREADS, 0, s>>>(F, L, g, fc, tape, stride, scales, ip, det,
                                                       det2, seeds, face_blocks, det_blocks);
    return cudaGetLastError();
  });
}

// Batched designs: njobs jobs of a list in device memory, max_blocks value
// blocks (record: per face; restore: faces and detectors) for the largest.
cudaError_t launch_record_batch(int dtype, const RecordJob* jobs, int njobs, int max_blocks,
                                cudaStream_t s) {
  if (njobs <= 0 || max_blocks <= 0) return cudaSuccess;
  return with_dtype(dtype, [&](auto dt) {
    constexpr int DT = decltype(dt)::value;
    k_record_flat_batch<DT><<<dim3(max_blocks, 6, njobs), FLAT_THREADS, 0, s>>>(jobs);
    return cudaGetLastError();
  });
}

cudaError_t launch_restore_seed_batch(int dtype, const RestoreJob* jobs, int njobs,
                                      int max_blocks, cudaStream_t s) {
  if (njobs <= 0 || max_blocks <= 0) return cudaSuccess;
  return with_dtype(dtype, [&](auto dt) {
    constexpr int DT = decltype(dt)::value;
    k_restore_seed_batch<DT><<<dim3(max_blocks, njobs), FLAT_THREADS, 0, s>>>(jobs);
    return cudaGetLastError();
  });
}

// The value and detector blocks of one restore launch (as launch_restore_seed counts them).
void restore_blocks(const Faces& fc, const Det& det, const Det& det2, int* face_blocks,
                    int* det_blocks) {
  *face_blocks = (fc.start[6] + FLAT_THREADS - 1) / FLAT_THREADS;
  int dmax = det.kind ? (det.u1 - det.u0) * (det.v1 - det.v0) : 0;
  if (det2.kind) dmax = max(dmax, (det2.u1 - det2.u0) * (det2.v1 - det2.v0));
  *det_blocks = (dmax + FLAT_THREADS - 1) / FLAT_THREADS;
}

int record_flat_blocks(const Faces& fc) {
  int m = 0;
  for (int f = 0; f < 6; ++f) m = max(m, (2 * fc.f[f].nu * fc.f[f].nv + FLAT_THREADS - 1) / FLAT_THREADS);
  return m;
}

// -------------------------------------------------------- raw codec ------
// One cluster of CTAs reduces the absmax of the whole array (test entry).
template <int DT>
__global__ void __launch_bounds__(REC_THREADS) k_encode(const float* __restrict__ in, size_t n,
                                                        void* code, float* scale_out,
                                                        int scaled) {
  typedef typename Code<DT>::T T;
  __shared__ float red[REC_THREADS / 32];
  __shared__ float cl_amax;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int nr = (int)cluster.num_blocks();
  const int tid = threadIdx.x;
  float scale = 1.0f;
  if (scaled) {
    float m = 0.f;
    for (size_t r = (size_t)rank * REC_THREADS + tid; r < n; r += (size_t)nr * REC_THREADS)
      m = fmaxf(m, fabsf(in[r]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    if (tid < 32) {
      float t = tid < REC_THREADS / 32 ? red[tid] : 0.f;
      for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
      if (tid == 0) cl_amax = t;
    }
    cluster.sync();
    float amax = 0.f;
    for (int b = 0; b < nr; ++b) amax = fmaxf(amax, *cluster.map_shared_rank(&cl_amax, b));
    cluster.sync();
    scale = amax > 0.f ? fmaxf(__fdiv_rn(amax, Code<DT>::fmax), kMinScale) : 1.0f;
  }
  if (rank == 0 && tid == 0) *scale_out = scale;
  T* out = reinterpret_cast<T*>(code);
  for (size_t r = (size_t)rank * REC_THREADS + tid; r < n; r += (size_t)nr * REC_THREADS)
    out[r] = Code<DT>::enc(scaled ? __fdiv_rn(in[r], scale) : in[r]);
}

template <int DT>
__global__ void k_decode(const void* code, size_t n, const float* scale, float* out) {
  typedef typename Code<DT>::T T;
  const T* c = reinterpret_cast<const T*>(code);
  float s = *scale;
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < n;
       r += (size_t)gridDim.x * blockDim.x)
    out[r] = Code<DT>::dec(c[r]) * s;
}

template <int DT>
static cudaError_t launch_encode_t(int scaled, const float* in, size_t n, void* code, float* scale,
                                   cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(REC_CLUSTER, 1, 1);
  cfg.blockDim = dim3(REC_THREADS, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = REC_CLUSTER;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_encode<DT>, in, n, code, scale, scaled);
}

cudaError_t launch_encode(int dtype, int scaled, const float* in, size_t n, void* code,
                          float* scale, cudaStream_t s) {
  return with_dtype(dtype, [&](auto dt) {
    constexpr int DT = decltype(dt)::value;
    return launch_encode_t<DT>(DT >= 2 ? scaled : 0, in, n, code, scale, s);
  });
}

cudaError_t launch_decode(int dtype, const void* code, size_t n, const float* scale, float* out,
                          cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  return with_dtype(dtype, [&](auto dt) {
    constexpr int DT = decltype(dt)::value;
    k_decode<DT><<<blocks, 256, 0, s>>>(code, n, scale, out);
    return cudaGetLastError();
  });
}

}  // namespace fdtd
