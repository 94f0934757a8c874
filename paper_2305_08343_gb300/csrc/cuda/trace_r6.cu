// trace_r6.cu — culled traversal variants for R = 6 (object masks of
// 6^3 bits): {uncompressed, compressed} x {closest, any} x {global table,
// shared-memory factored table, bit table (compressed)} x {scales divided,
// scales stored}, the R_ray = 2R table (uncompressed, scales stored); and
// the wave pipeline kernels.  The factored tables of the wave pipeline and
// the L1-read factored tables are in trace_r6f.cu.
#include "trace_kernel.cuh"

namespace sct {

KernelFn get_kernel_r6f(int mode);
WaveKernelFn get_waves_r6f(int lutv, int block, int stack);

#define SCT_V(C, M, L) {trace_kernel<6, C, M, L, 0>, trace_kernel<6, C, M, L, 1>}
KernelFn get_kernel_r6(int cull, int mode, int lutv, int scales) {
  if (lutv == 5) return cull == 1 && scales ? get_kernel_r6f(mode) : nullptr;
  static const KernelFn unc[2][2][2] = {
      {SCT_V(1, 0, 0), SCT_V(1, 0, 1)}, {SCT_V(1, 1, 0), SCT_V(1, 1, 1)}};
  static const KernelFn comp[2][3][2] = {
      {SCT_V(2, 0, 0), SCT_V(2, 0, 1), SCT_V(2, 0, 2)},
      {SCT_V(2, 1, 0), SCT_V(2, 1, 1), SCT_V(2, 1, 2)}};
  if (cull == 1 && lutv == 4) return mode ? trace_kernel<6, 1, 1, 4, 1> : trace_kernel<6, 1, 0, 4, 1>;
  if (cull == 1) return unc[mode][lutv == 1 ? 1 : 0][scales];
  return comp[mode][lutv][scales];
}
#undef SCT_V

WaveKernelFn get_waves_r6(int cull, int lutv, int scales, int block, int stack) {
  if (cull == 1 && lutv == 4) return WaveVariants<6, 1, 4, 1>::get(block, stack);
  if (lutv == 5) return cull == 1 && scales ? get_waves_r6f(5, block, stack) : nullptr;
  // factored tables in shared memory: stored scales only (divided scales
  // keep the full table in the wave pipeline)
  if (cull == 1 && lutv == 1 && scales) return get_waves_r6f(1, block, stack);
  if (cull == 1)
    return scales ? WaveVariants<6, 1, 0, 1>::get(block, stack)
                  : WaveVariants<6, 1, 0, 0>::get(block, stack);
  if (lutv == 2)
    return scales ? WaveVariants<6, 2, 2, 1>::get(block, stack)
                  : WaveVariants<6, 2, 2, 0>::get(block, stack);
  if (block != kBlock || stack != kStack) return nullptr;
  return scales ? waves_kernel<6, 2, 0, 1> : waves_kernel<6, 2, 0, 0>;
}

SeededKernelFn get_seeded_r6(int cull, int lutv, int scales) {
  if (cull == 1 && lutv == 4) return seeded_kernel<6, 1, 4, 1>;
  if (cull == 1) return scales ? seeded_kernel<6, 1, 0, 1> : seeded_kernel<6, 1, 0, 0>;
  if (lutv == 2) return scales ? seeded_kernel<6, 2, 2, 1> : seeded_kernel<6, 2, 2, 0>;
  return scales ? seeded_kernel<6, 2, 0, 1> : seeded_kernel<6, 2, 0, 0>;
}

}  // namespace sct
