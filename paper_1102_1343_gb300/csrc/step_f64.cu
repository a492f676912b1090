// FP64 instantiation of the fire-step kernels (every field in double).
#include "march_kernel.cuh"
#include "step_kernel.cuh"
#include "warp_kernel.cuh"

namespace wf {
WF_INSTANTIATE(double)
WF_INSTANTIATE_MARCH(double)
WF_INSTANTIATE_WARP(double)
}  // namespace wf
