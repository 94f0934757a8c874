// trace_var.cu — kernels with non-default OPT bits (trace_kernel.cuh): the
// fused Alg. 1 cell form, and the load-scheduling, stack-placement and
// bounce-sort options, for the R = 6 images (uncompressed masks with the full table,
// compressed masks with the bit table) and the plain traversal, in the
// single-batch kernel and the wave pipeline (block 128, stack 64).
#include "trace_kernel.cuh"

namespace sct {

namespace {

template <int R, int CULL, int LUTV, int SCALES, int OPT>
KernelFn kernel_of(int mode) {
  return mode ? trace_kernel<R, CULL, 1, LUTV, SCALES, 2, OPT> : trace_kernel<R, CULL, 0, LUTV, SCALES, 2, OPT>;
}

template <int R, int CULL, int LUTV, int SCALES, int OPT>
WaveKernelFn waves_of() {
  return waves_kernel<R, CULL, LUTV, SCALES, kBlock, kStack, 2, OPT>;
}

// The option sets built here.
#define SCT_OPTS(X)                                                                   \
  X(OPT_FUSED) X(OPT_PAIR) X(OPT_SPEC) X(OPT_TOS) X(OPT_SPEC | OPT_TOS) X(OPT_SORT) \
  X(OPT_SPEC | OPT_TOS | OPT_SORT) X(OPT_FUSED | OPT_SPEC | OPT_TOS | OPT_SORT) X(OPT_DEFER) \
  X(OPT_LAZY) X(OPT_SSTACK) X(OPT_TL1) X(OPT_OCC9) X(OPT_OCC9 | OPT_SSTACK) X(OPT_OCC10) \
  X(OPT_OCC10 | OPT_SSTACK) X(OPT_HSLOT) X(OPT_HSLOT | OPT_OCC9) X(OPT_HSLOT | OPT_OCC9 | OPT_SSTACK)

}  // namespace

bool var_supported(int opt) {
#define SCT_CASE(O) if (opt == (O)) return true;
  SCT_OPTS(SCT_CASE)
#undef SCT_CASE
  return false;
}

// R = 6: cull 1 (uncompressed, full table, lutv 0) or 2 (compressed, bit
// table, lutv 2), scales stored; R = 0: plain.  nullptr if not built.
KernelFn get_kernel_var(int R, int cull, int mode, int lutv, int opt) {
#define SCT_CASE(O)                                                        \
  if (opt == (O)) {                                                        \
    if (R == 0) return kernel_of<0, 0, 0, 0, (O) & ~OPT_DEFER>(mode);      \
    if (cull == 1 && lutv == 0) return kernel_of<6, 1, 0, 1, (O) & ~OPT_DEFER>(mode); \
    if (cull == 2 && lutv == 2) return kernel_of<6, 2, 2, 1, (O)>(mode);   \
    return nullptr;                                                        \
  }
  SCT_OPTS(SCT_CASE)
#undef SCT_CASE
  return nullptr;
}

WaveKernelFn get_waves_var(int R, int cull, int lutv, int opt) {
#define SCT_CASE(O)                                                   \
  if (opt == (O)) {                                                   \
    if (R == 0) return waves_of<0, 0, 0, 0, (O) & ~OPT_DEFER>();      \
    if (cull == 1 && lutv == 0) return waves_of<6, 1, 0, 1, (O) & ~OPT_DEFER>(); \
    if (cull == 2 && lutv == 2) return waves_of<6, 2, 2, 1, (O)>();   \
    return nullptr;                                                   \
  }
  SCT_OPTS(SCT_CASE)
#undef SCT_CASE
  return nullptr;
}

}  // namespace sct
