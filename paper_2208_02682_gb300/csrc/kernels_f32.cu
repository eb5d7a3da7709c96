// FP32 instantiation of the stage kernels and their launchers.
#define LM_INSTANTIATE
#include "launch.cuh"

namespace lm {
LM_INSTANTIATE_ALL(float)

cudaError_t prepare_kernels_f32() {
  cudaError_t e = prepare_kernels_t<float>();
  if (e != cudaSuccess) return e;
  int dev = 0, mx = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  if ((e = allow_dynamic_smem(k_stage_col_fwd_pipe<10>, mx)) != cudaSuccess) return e;
  return allow_dynamic_smem(k_stage_col_fwd_pipe<11>, mx);
}

cudaError_t launch_col_fwd_pipe(int L, const RunDesc<float>* runs, const int* start, int nruns, int blocks,
                                int threads, size_t smem, int total, bool pdl, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  if (L == 10) return cudaLaunchKernelEx(&cfg, k_stage_col_fwd_pipe<10>, runs, start, nruns, total);
  if (L == 11) return cudaLaunchKernelEx(&cfg, k_stage_col_fwd_pipe<11>, runs, start, nruns, total);
  return cudaErrorInvalidValue;
}

int col_fwd_pipe_occupancy(int L, int threads, size_t smem) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (L == 10) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage_col_fwd_pipe<10>, threads, smem);
  if (L == 11) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage_col_fwd_pipe<11>, threads, smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}
}  // namespace lm
