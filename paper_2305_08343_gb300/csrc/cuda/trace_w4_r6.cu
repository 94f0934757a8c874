// trace_w4_r6.cu — culled traversal on 4-wide nodes (SC_LAYOUT_MASKED4) at
// R = 6: {uncompressed, compressed} x {closest, any} x {global table, bit
// table (compressed)}, scales stored; wave kernels with blocks of 128 / 256
// threads and a 64-entry stack.
#include "trace_kernel.cuh"

namespace sct {

KernelFn get_kernel_w4_r6(int cull, int mode, int lutv) {
  static const KernelFn unc[2] = {trace_kernel<6, 1, 0, 0, 1, 4>, trace_kernel<6, 1, 1, 0, 1, 4>};
  static const KernelFn comp[2][2] = {
      {trace_kernel<6, 2, 0, 0, 1, 4>, trace_kernel<6, 2, 0, 2, 1, 4>},
      {trace_kernel<6, 2, 1, 0, 1, 4>, trace_kernel<6, 2, 1, 2, 1, 4>}};
  if (cull == 1) return unc[mode];
  return comp[mode][lutv == 2 ? 1 : 0];
}

WaveKernelFn get_waves_w4_r6(int cull, int lutv, int block) {
  static const WaveKernelFn unc[2] = {waves_kernel<6, 1, 0, 1, 128, 64, 4>,
                                      waves_kernel<6, 1, 0, 1, 256, 64, 4>};
  static const WaveKernelFn comp[2][2] = {
      {waves_kernel<6, 2, 0, 1, 128, 64, 4>, waves_kernel<6, 2, 0, 1, 256, 64, 4>},
      {waves_kernel<6, 2, 2, 1, 128, 64, 4>, waves_kernel<6, 2, 2, 1, 256, 64, 4>}};
  const int b = block == 256 ? 1 : 0;
  if (cull == 1) return unc[b];
  return comp[lutv == 2 ? 1 : 0][b];
}

}  // namespace sct
