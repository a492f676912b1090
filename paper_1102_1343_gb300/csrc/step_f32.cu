// FP32 instantiation of the fire-step kernels (float state, double ignition
// time and heat reduction).
#include "march_kernel.cuh"
#include "step_kernel.cuh"
#include "warp_kernel.cuh"

namespace wf {
WF_INSTANTIATE(float)
WF_INSTANTIATE_MARCH(float)
WF_INSTANTIATE_WARP(float)
}  // namespace wf
