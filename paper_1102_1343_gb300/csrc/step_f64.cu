// FP64 instantiation of the fire-step kernels (every field in double).
#include "step_kernel.cuh"

namespace wf {
WF_INSTANTIATE(double)
}  // namespace wf
