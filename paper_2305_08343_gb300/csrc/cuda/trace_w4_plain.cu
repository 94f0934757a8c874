// trace_w4_plain.cu — plain traversal on 4-wide nodes (SC_LAYOUT_PLAIN4 or
// a masked 4-wide image traced without culling): closest / any hit; wave
// kernels with blocks of 128 / 256 threads and a 64-entry stack.
#include "trace_kernel.cuh"

namespace sct {

KernelFn get_kernel_w4_plain(int mode) {
  return mode ? trace_kernel<0, 0, 1, 0, 0, 4> : trace_kernel<0, 0, 0, 0, 0, 4>;
}

WaveKernelFn get_waves_w4_plain(int block) {
  return block == 256 ? waves_kernel<0, 0, 0, 0, 256, 64, 4> : waves_kernel<0, 0, 0, 0, 128, 64, 4>;
}

}  // namespace sct
