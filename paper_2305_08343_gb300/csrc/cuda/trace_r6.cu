// trace_r6.cu — culled traversal variants for R = 6 (object masks of
// 6^3 bits): {uncompressed, compressed} x {closest, any} x {global table,
// shared-memory factored table}.
#include "trace_kernel.cuh"

namespace sct {

KernelFn get_kernel_r6(int cull, int mode, int lutv) {
  static const KernelFn table[2][2][2] = {
      {{trace_kernel<6, 1, 0, 0>, trace_kernel<6, 1, 0, 1>},
       {trace_kernel<6, 1, 1, 0>, trace_kernel<6, 1, 1, 1>}},
      {{trace_kernel<6, 2, 0, 0>, trace_kernel<6, 2, 0, 1>},
       {trace_kernel<6, 2, 1, 0>, trace_kernel<6, 2, 1, 1>}}};
  return table[cull - 1][mode][lutv];
}

}  // namespace sct
