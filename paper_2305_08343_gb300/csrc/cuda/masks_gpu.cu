// masks_gpu.cu — the object masks of every child slot built on the GPU
// (sc_build_opts.gpu_masks): the same per-voxel and per-cell computation as
// the host builder (host/mask_math.h, one source), one warp per child slot,
// the levels of the tree processed from the deepest so that each level
// reads only finished masks of deeper nodes.  The bits are identical to the
// host build's.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "host/internal.h"
#include "host/mask_math.h"

namespace sc {
namespace {

// One warp per child slot: the lanes split each triangle's candidate voxels
// (SAT tests) and each descendant's child cells (Alg. 2 fill), each lane
// collecting bits in its own copy of the mask, OR-reduced at the end.  The
// per-voxel and per-cell arithmetic is mask_math.h's, so the bits are those
// of the host build.
// Per-warp tables of the FP32 SAT filter: the half extents of the slot's
// voxels per axis and index (set once per slot), and each vertex coordinate
// of the current triangle relative to every voxel centre on its axis (set
// once per triangle), so that a triangle/voxel pair needs no FP64 work
// unless the filter leaves it undecided.
// Threads per block of slot_masks_kernel: one warp per child slot, and
// one set of shared-memory tables per warp.
constexpr int kMaskThreads = 128;
constexpr int kMaskWarps = kMaskThreads / 32;

struct SatTables {
  mm::Ef h[3][8];
  mm::Ef a[3][3][8];  // [vertex][axis][voxel index]
  int fill_lo[3][9], fill_hi[3][9];  // Alg. 2 parent ranges of the current fill
};

__device__ void voxelize_warp(const float* t9, const mm::Grid& g, uint32_t* acc, int W,
                              int lane, SatTables& tab) {
  double v[9];
  for (int i = 0; i < 9; ++i) v[i] = (double)t9[i];
  // the candidate range of axis k is found by lane k and broadcast
  int c0 = 0, c1 = 0;
  if (lane < 3) {
    const int k = lane;
    const double tlo = mm::mn(mm::mn(v[k], v[3 + k]), v[6 + k]);
    const double thi = mm::mx(mm::mx(v[k], v[3 + k]), v[6 + k]);
    g.candidates(k, tlo, thi, c0, c1);
  }
  int r0[3], r1[3];
  for (int k = 0; k < 3; ++k) {
    r0[k] = __shfl_sync(0xffffffffu, c0, k);
    r1[k] = __shfl_sync(0xffffffffu, c1, k);
  }
  const int R = g.R, nx = r1[0] - r0[0] + 1, ny = r1[1] - r0[1] + 1, nz = r1[2] - r0[2] + 1;
  __syncwarp();  // the previous triangle's table has been read
  for (int idx = lane; idx < 9 * R; idx += 32) {
    const int i = idx / (3 * R), k = (idx / R) % 3, j = idx % R;
    tab.a[i][k][j] = mm::ef_rel(v[3 * i + k], g.b0[k][j], g.b1[k][j]);
  }
  __syncwarp();
  // voxels an earlier triangle set need no test (the bits are an OR)
  uint32_t have[16];
  for (int w = 0; w < W; ++w) have[w] = __reduce_or_sync(0xffffffffu, acc[w]);
  for (int i = lane; i < nx * ny * nz; i += 32) {
    const int x = r0[0] + i % nx, y = r0[1] + (i / nx) % ny, z = r0[2] + i / (nx * ny);
    if (mm::get_bit(have, x + R * y + R * R * z)) continue;
    const mm::Ef a[3][3] = {{tab.a[0][0][x], tab.a[0][1][y], tab.a[0][2][z]},
                            {tab.a[1][0][x], tab.a[1][1][y], tab.a[1][2][z]},
                            {tab.a[2][0][x], tab.a[2][1][y], tab.a[2][2][z]}};
    const mm::Ef h[3] = {tab.h[0][x], tab.h[1][y], tab.h[2][z]};
    int hit = mm::tri_box_overlap_ef(a, h);
    if (hit < 0) {
      const double bmin[3] = {g.b0[0][x], g.b0[1][y], g.b0[2][z]};
      const double bmax[3] = {g.b1[0][x], g.b1[1][y], g.b1[2][z]};
      hit = mm::tri_box_overlap(v, bmin, bmax) ? 1 : 0;
    }
    if (hit) mm::set_bit(acc, x + R * y + R * R * z);
  }
}

// Alg. 2 fill of one descendant's mask: the parent ranges of the 3 (R + 1)
// child borders are computed one per lane (R + 1 <= 9) into the warp's
// table, then the lanes split the child's set cells.
__device__ void fill_warp(uint32_t* acc, const float* pbox, const uint32_t* cmask,
                          const float* cbox, int R, double eps, int lane, SatTables& tab) {
  __syncwarp();  // the previous fill's table has been read
  if (lane < 3 * (R + 1)) {
    const int k = lane / (R + 1), i = lane % (R + 1);
    mm::fill_range(pbox, cbox, k, i, R, eps, tab.fill_lo[k][i], tab.fill_hi[k][i]);
  }
  __syncwarp();
  const int(*lo_i)[9] = tab.fill_lo;
  const int(*hi_i)[9] = tab.fill_hi;
  for (int cell = lane; cell < R * R * R; cell += 32) {
    if (!mm::get_bit(cmask, cell)) continue;
    const int x = cell % R, y = (cell / R) % R, z = cell / (R * R);
    for (int pz = lo_i[2][z]; pz <= hi_i[2][z + 1]; ++pz)
      for (int py = lo_i[1][y]; py <= hi_i[1][y + 1]; ++py)
        for (int px = lo_i[0][x]; px <= hi_i[0][x + 1]; ++px)
          mm::set_bit(acc, px + R * py + R * R * pz);
  }
}

__device__ void leaf_warp(const mm::MaskInputs& b, int32_t first, int32_t count,
                          const mm::Grid& g, uint32_t* acc, int lane, SatTables& tab) {
  for (int32_t i = 0; i < count; ++i)
    voxelize_warp(&b.tris[9 * (size_t)b.perm[first + i]], g, acc, b.W, lane, tab);
}

__global__ void slot_masks_kernel(mm::MaskInputs in, const int64_t* nodes, int64_t nslots) {
  const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (slot >= nslots) return;  // uniform across the warp
  const int64_t n = nodes[slot >> 1];
  const int c = (int)(slot & 1);
  const float* gbox = &in.box[12 * n + 6 * c];
  // the slot's grid, built entry by entry by the lanes of the warp (the
  // same operations as Grid::init) in shared memory
  __shared__ mm::Grid grids[kMaskWarps];
  __shared__ SatTables tables[kMaskWarps];
  const int wib = threadIdx.x >> 5;
  mm::Grid& g = grids[wib];
  SatTables& tab = tables[wib];
  if (lane == 0) {
    g.R = in.R;
    g.eps = in.eps;
  }
  if (lane < 3) g.init_axis(gbox, lane);
  __syncwarp();
  if (lane < 3 * in.R) g.init_cell(lane / in.R, lane % in.R);
  __syncwarp();
  for (int idx = lane; idx < 3 * in.R; idx += 32) {
    const int k = idx / in.R, j = idx % in.R;
    tab.h[k][j] = mm::ef_half_extent(g.b0[k][j], g.b1[k][j]);
  }
  __syncwarp();
  uint32_t acc[16];
  for (int w = 0; w < 16; ++w) acc[w] = 0u;
  const int32_t ch = in.child[2 * n + c], cn = in.count[2 * n + c];
  if (cn > 0) {
    leaf_warp(in, ch, cn, g, acc, lane, tab);
  } else {
    // the descendants of mm::collect, visited in the same order by every lane
    int64_t node[mm::kMaxL];
    int depth[mm::kMaxL], next[mm::kMaxL];
    int sp = 0;
    node[0] = ch;
    depth[0] = 1;
    next[0] = 0;
    while (sp >= 0) {
      if (next[sp] == 2) {
        --sp;
        continue;
      }
      const int64_t m = node[sp];
      const int cc = next[sp]++;
      const int32_t mch = in.child[2 * m + cc], mcn = in.count[2 * m + cc];
      const float* cbox = &in.box[12 * m + 6 * cc];
      if (depth[sp] == in.L) {
        fill_warp(acc, gbox, &in.masks[((size_t)m * 2 + cc) * in.W], cbox, in.R, in.eps, lane,
                  tab);
      } else if (mcn > 0) {
        leaf_warp(in, mch, mcn, g, acc, lane, tab);
      } else {
        node[sp + 1] = mch;
        depth[sp + 1] = depth[sp] + 1;
        next[sp + 1] = 0;
        ++sp;
      }
    }
  }
  uint32_t* out = &in.masks[((size_t)n * 2 + c) * in.W];
  for (int w = 0; w < in.W; ++w) {
    const uint32_t v = __reduce_or_sync(0xffffffffu, acc[w]);
    if (lane == 0) out[w] = v;
  }
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

namespace {

// The masks of every node (node_dirty NULL: b.masks starts at zero) or of
// the marked nodes only (the other masks are uploaded and kept), level by
// level from the deepest.  Uses b.R, b.L, b.W, b.eps.
void masks_gpu_levels(Bvh& b, const std::vector<uint8_t>* node_dirty) {
  const int L = b.L;
  if (std::min(L, b.max_depth + 1) > mm::kMaxL)
    fail(SC_ERR_UNSUPPORTED, "mask depth L = %d over a tree %d deep exceeds %d", L,
         b.max_depth, mm::kMaxL);
  std::vector<std::vector<int64_t>> levels(b.max_depth + 1);
  for (int64_t n = 0; n < b.nn; ++n)
    if (!node_dirty || (*node_dirty)[n]) levels[b.ndepth[n]].push_back(n);
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
  if (node_dirty) {
    in.masks = upload(d, b.masks, st);
  } else {
    in.masks = d.alloc<uint32_t>(b.masks.size());
    CUDA_OK(cudaMemsetAsync(in.masks, 0, b.masks.size() * sizeof(uint32_t), st));
  }
  in.R = b.R;
  in.L = std::min(L, b.max_depth + 1);
  in.W = b.W;
  in.eps = b.eps;
  const int64_t* d_order = upload(d, order, st);
  for (int dep = b.max_depth; dep >= 0; --dep) {
    const int64_t nslots = 2 * (int64_t)(start[dep + 1] - start[dep]);
    if (nslots == 0) continue;
    const int threads = kMaskThreads;  // a warp per slot
    const int64_t warps_per_block = threads / 32;
    slot_masks_kernel<<<(unsigned)((nslots + warps_per_block - 1) / warps_per_block), threads, 0,
                        st>>>(in, d_order + start[dep], nslots);
    CUDA_OK(cudaGetLastError());
  }
  CUDA_OK(cudaMemcpyAsync(b.masks.data(), in.masks, b.masks.size() * sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, st));
  CUDA_OK(cudaStreamSynchronize(st));
}

}  // namespace

void build_masks_gpu(Bvh& b, int R, int L, double eps) {
  const double t0 = now_ms();
  b.R = R;
  b.L = L;
  b.W = mask_words(R);
  b.eps = eps;
  b.masks.assign((size_t)b.nn * 2 * b.W, 0u);
  if (b.nn > 0) masks_gpu_levels(b, nullptr);
  b.ms_masks = now_ms() - t0;
}

void refit_masks_gpu(Bvh& b, const std::vector<uint8_t>& node_dirty) {
  const double t0 = now_ms();
  if (b.nn > 0) masks_gpu_levels(b, &node_dirty);
  b.ms_masks = now_ms() - t0;
}

}  // namespace sc
