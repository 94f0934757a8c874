// masks_gpu.cu — the object masks of every child slot built on the GPU
// (sc_build_opts.gpu_masks): the same per-slot computation as the host
// builder (host/mask_math.h, one source), one thread per child slot, the
// levels of the tree processed from the deepest so that each level reads
// only finished masks of deeper nodes.  The bits are identical to the host
// build's.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "host/internal.h"
#include "host/mask_math.h"

namespace sc {
namespace {

__global__ void slot_masks_kernel(mm::MaskInputs in, const int64_t* nodes, int64_t nslots) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nslots) return;
  mm::slot_mask(in, nodes[i >> 1], (int)(i & 1));
}

#define CUDA_OK(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      fail(SC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

// Device buffers freed on every exit path.
struct DevBufs {
  std::vector<void*> ptrs;
  template <class T>
  T* alloc(size_t n) {
    void* p = nullptr;
    CUDA_OK(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)));
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~DevBufs() {
    for (void* p : ptrs) cudaFree(p);
  }
};

template <class T>
T* upload(DevBufs& d, const std::vector<T>& v, cudaStream_t st) {
  T* p = d.alloc<T>(v.size());
  if (!v.empty()) CUDA_OK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return p;
}

}  // namespace

void build_masks_gpu(Bvh& b, int R, int L, double eps) {
  const double t0 = now_ms();
  b.R = R;
  b.L = L;
  b.W = mask_words(R);
  b.eps = eps;
  b.masks.assign((size_t)b.nn * 2 * b.W, 0u);
  if (b.nn == 0) {
    b.ms_masks = now_ms() - t0;
    return;
  }
  if (std::min(L, b.max_depth + 1) > mm::kMaxL)
    fail(SC_ERR_UNSUPPORTED, "mask depth L = %d over a tree %d deep exceeds %d", L,
         b.max_depth, mm::kMaxL);
  std::vector<std::vector<int64_t>> levels(b.max_depth + 1);
  for (int64_t n = 0; n < b.nn; ++n) levels[b.ndepth[n]].push_back(n);
  std::vector<int64_t> order;
  std::vector<size_t> start(b.max_depth + 2, 0);
  for (int d = 0; d <= b.max_depth; ++d) {
    start[d] = order.size();
    order.insert(order.end(), levels[d].begin(), levels[d].end());
  }
  start[b.max_depth + 1] = order.size();
  cudaStream_t st = nullptr;
  CUDA_OK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } guard{st};
  DevBufs d;
  mm::MaskInputs in;
  in.tris = upload(d, b.tris, st);
  in.perm = upload(d, b.perm, st);
  in.child = upload(d, b.child, st);
  in.count = upload(d, b.count, st);
  in.box = upload(d, b.box, st);
  in.masks = d.alloc<uint32_t>(b.masks.size());
  CUDA_OK(cudaMemsetAsync(in.masks, 0, b.masks.size() * sizeof(uint32_t), st));
  in.R = R;
  in.L = std::min(L, b.max_depth + 1);
  in.W = b.W;
  in.eps = eps;
  const int64_t* d_order = upload(d, order, st);
  for (int dep = b.max_depth; dep >= 0; --dep) {
    const int64_t nslots = 2 * (int64_t)(start[dep + 1] - start[dep]);
    if (nslots == 0) continue;
    const int threads = 128;
    slot_masks_kernel<<<(unsigned)((nslots + threads - 1) / threads), threads, 0, st>>>(
        in, d_order + start[dep], nslots);
    CUDA_OK(cudaGetLastError());
  }
  CUDA_OK(cudaMemcpyAsync(b.masks.data(), in.masks, b.masks.size() * sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, st));
  CUDA_OK(cudaStreamSynchronize(st));
  b.ms_masks = now_ms() - t0;
}

}  // namespace sc
