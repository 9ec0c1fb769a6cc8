// Instantiations of the MP loop kernel: FP32 planes.
#include "mp_loop_kernel.cuh"

namespace mpg {
LoopKernel_t loop_kernel_f32(int threads, bool pow2) { return loop_kernel_t<float2>(threads, pow2); }
}  // namespace mpg
