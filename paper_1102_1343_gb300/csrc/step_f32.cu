// FP32 instantiation of the fire-step kernels (float state, double ignition
// time and heat reduction).
#include "step_kernel.cuh"

namespace wf {
WF_INSTANTIATE(float)
}  // namespace wf
