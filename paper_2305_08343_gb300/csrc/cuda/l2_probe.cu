// l2_probe.cu — L2 read bandwidth probe: the roofline denominator for work
// whose data stays in the 129 MB L2 (the traversal of a scene whose BVH fits
// there).  Every thread of a full grid reads 16-byte words of the buffer
// through L2 only (ld.global.cg, no L1 allocation), `reps` passes, and XORs
// them together; each block folds its threads' values into one sink word, so
// that no load can be dropped.
#include <cuda_runtime.h>

#include <cstdint>

#include "host/internal.h"

namespace sc {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;

__global__ void __launch_bounds__(kProbeThreads)
    l2_read_kernel(const uint4* __restrict__ buf, size_t n16, int reps,
                   unsigned long long* __restrict__ sink) {
  __shared__ unsigned int fold;
  if (threadIdx.x == 0) fold = 0u;
  __syncthreads();
  unsigned int acc = 0u;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
      const uint4 v = __ldcg(buf + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  atomicXor(&fold, acc);
  __syncthreads();
  if (threadIdx.x == 0) sink[blockIdx.x] = fold;
}

int probe_blocks() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms * kProbeBlocksPerSm;
}

}  // namespace
}  // namespace sc

using namespace sc;

extern "C" {

int sc_l2_probe_blocks(void) { return probe_blocks(); }

sc_status sc_l2_read(const void* d_buf, size_t bytes, int reps, uint64_t* d_sink,
                     void* stream) {
  try {
    clear_error();
    if (!d_buf || !d_sink) fail(SC_ERR_ARG, "sc_l2_read: NULL buffer");
    if ((reinterpret_cast<uintptr_t>(d_buf) & 15) || (bytes & 15) || bytes == 0)
      fail(SC_ERR_ARG, "sc_l2_read: the buffer must be 16-byte aligned, a multiple of 16 bytes");
    if (reps < 1) fail(SC_ERR_ARG, "sc_l2_read: reps must be >= 1");
    const int blocks = probe_blocks();
    if (blocks <= 0) fail(SC_ERR_CUDA, "sc_l2_read: no CUDA device");
    l2_read_kernel<<<blocks, kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint4*>(d_buf), bytes / 16, reps,
        reinterpret_cast<unsigned long long*>(d_sink));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(SC_ERR_CUDA, "sc_l2_read: %s", cudaGetErrorString(e));
    return SC_OK;
  } catch (const Error& e) {
    set_error("%s", e.msg.c_str());
    return e.code;
  }
}

}  // extern "C"
