// trace_plain.cu — unculled traversal (the baseline the culling is measured
// against): same kernel, same node records, no mask test.
#include "trace_kernel.cuh"

namespace sct {

KernelFn get_kernel_plain(int mode) {
  return mode ? trace_kernel<0, 0, 1, 0, 0> : trace_kernel<0, 0, 0, 0, 0>;
}

WaveKernelFn get_waves_plain(int block, int stack) {
  return WaveVariants<0, 0, 0, 0>::get(block, stack);
}

SeededKernelFn get_seeded_plain() { return seeded_kernel<0, 0, 0, 0>; }

}  // namespace sct
