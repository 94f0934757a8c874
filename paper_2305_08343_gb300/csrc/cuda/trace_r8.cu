// trace_r8.cu — culled traversal variants for R = 8 (object masks of
// 8^3 bits): {uncompressed, compressed} x {closest, any} x {global table,
// shared-memory factored table}.
#include "trace_kernel.cuh"

namespace sct {

KernelFn get_kernel_r8(int cull, int mode, int lutv) {
  static const KernelFn table[2][2][2] = {
      {{trace_kernel<8, 1, 0, 0>, trace_kernel<8, 1, 0, 1>},
       {trace_kernel<8, 1, 1, 0>, trace_kernel<8, 1, 1, 1>}},
      {{trace_kernel<8, 2, 0, 0>, trace_kernel<8, 2, 0, 1>},
       {trace_kernel<8, 2, 1, 0>, trace_kernel<8, 2, 1, 1>}}};
  return table[cull - 1][mode][lutv];
}

}  // namespace sct
