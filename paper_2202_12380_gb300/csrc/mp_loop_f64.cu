// Instantiations of the MP loop kernel: FP64 planes (MP_COEF_FP64).
#include "mp_loop_kernel.cuh"

namespace mpg {
LoopKernel_t loop_kernel_f64(int threads, bool pow2) { return loop_kernel_t<double2>(threads, pow2); }
}  // namespace mpg
