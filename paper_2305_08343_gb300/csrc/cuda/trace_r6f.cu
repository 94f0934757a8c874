// trace_r6f.cu — culled traversal for R = 6 images with uncompressed masks
// and stored scales, with the ray mask taken from the factored 2-D tables
// (Helly's theorem on the t-intervals): staged in shared memory (lookup
// variant 1, wave pipeline) or read through L1 from the image (lookup
// variant 5, single-batch kernel and wave pipeline).
#include "trace_kernel.cuh"

namespace sct {

KernelFn get_kernel_r6f(int mode) {
  return mode ? trace_kernel<6, 1, 1, 5, 1> : trace_kernel<6, 1, 0, 5, 1>;
}

WaveKernelFn get_waves_r6f(int lutv, int block, int stack) {
  return lutv == 5 ? WaveVariants<6, 1, 5, 1>::get(block, stack)
                   : WaveVariants<6, 1, 1, 1>::get(block, stack);
}

}  // namespace sct
