// The four-column warp-marching step kernel (FP32 only): its own translation
// unit, so that it compiles in parallel with the others.
#include "warp4_kernel.cuh"
