// FP32 instantiation of the stage kernels and their launchers.
#define LM_INSTANTIATE
#include "launch.cuh"

namespace lm {
LM_INSTANTIATE_ALL(float)
cudaError_t prepare_kernels_f32() { return prepare_kernels_t<float>(); }
}  // namespace lm
