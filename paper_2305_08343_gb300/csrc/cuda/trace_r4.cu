// trace_r4.cu — culled traversal variants for R = 4 (object masks of 64
// bits): {uncompressed, compressed} x {closest, any} x {global table,
// shared table, bit table (compressed)} x {scales divided, scales stored},
// the R_ray = 2R table (uncompressed, scales stored); and the wave pipeline
// kernels.  At R = 4 the "shared" lookup stages the
// whole ray-mask table (32 KB) and the compression LUT in shared memory.
#include "trace_kernel.cuh"

namespace sct {

#define SCT_V(C, M, L) {trace_kernel<4, C, M, L, 0>, trace_kernel<4, C, M, L, 1>}
KernelFn get_kernel_r4(int cull, int mode, int lutv, int scales) {
  static const KernelFn unc[2][2][2] = {
      {SCT_V(1, 0, 0), SCT_V(1, 0, 3)}, {SCT_V(1, 1, 0), SCT_V(1, 1, 3)}};
  static const KernelFn comp[2][3][2] = {
      {SCT_V(2, 0, 0), SCT_V(2, 0, 3), SCT_V(2, 0, 2)},
      {SCT_V(2, 1, 0), SCT_V(2, 1, 3), SCT_V(2, 1, 2)}};
  if (cull == 1 && lutv == 4) return mode ? trace_kernel<4, 1, 1, 4, 1> : trace_kernel<4, 1, 0, 4, 1>;
  if (cull == 1) return unc[mode][lutv == 1 ? 1 : 0][scales];
  return comp[mode][lutv][scales];
}
#undef SCT_V

WaveKernelFn get_waves_r4(int cull, int lutv, int scales) {
  static const WaveKernelFn unc[2][2] = {
      {waves_kernel<4, 1, 0, 0>, waves_kernel<4, 1, 0, 1>},
      {waves_kernel<4, 1, 3, 0>, waves_kernel<4, 1, 3, 1>}};
  static const WaveKernelFn comp[3][2] = {
      {waves_kernel<4, 2, 0, 0>, waves_kernel<4, 2, 0, 1>},
      {waves_kernel<4, 2, 3, 0>, waves_kernel<4, 2, 3, 1>},
      {waves_kernel<4, 2, 2, 0>, waves_kernel<4, 2, 2, 1>}};
  if (cull == 1 && lutv == 4) return waves_kernel<4, 1, 4, 1>;
  if (cull == 1) return unc[lutv == 1 ? 1 : 0][scales];
  return comp[lutv][scales];
}

SeededKernelFn get_seeded_r4(int cull, int lutv, int scales) {
  if (cull == 1 && lutv == 4) return seeded_kernel<4, 1, 4, 1>;
  if (cull == 1) return scales ? seeded_kernel<4, 1, 0, 1> : seeded_kernel<4, 1, 0, 0>;
  if (lutv == 2) return scales ? seeded_kernel<4, 2, 2, 1> : seeded_kernel<4, 2, 2, 0>;
  return scales ? seeded_kernel<4, 2, 0, 1> : seeded_kernel<4, 2, 0, 0>;
}

}  // namespace sct
