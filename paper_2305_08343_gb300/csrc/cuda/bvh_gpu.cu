// bvh_gpu.cu — the binned-SAH BVH2 of bvh_build.cpp built on the GPU
// (sc_build_opts.gpu_bvh).  It follows the same canonical rule set
// (triangle boxes and double centroids, the bin index, the greedy Eq. 1
// cost, ties to the lower axis then the lower plane, the half split when no
// plane is valid, a stable partition, pre-order numbering), so the tree --
// node numbering, child boxes, leaf ranges and triangle order -- is the host
// build's.  Every reduction is a min/max or an integer count, which no
// order of evaluation changes (a zero bound may differ in sign only).
//
// Two phases:
//  * ranges of more than kTaskMax triangles are split level by level by
//    grid-wide kernels over fixed-size chunks of the triangle order (range
//    statistics, bins, one warp per range for the cost sweep, counting, and a
//    stable scatter), with one small host round trip per level;
//  * every smaller range is a task: one warp builds its whole subtree, the
//    ranges taken depth first (left before right), so its nodes come out in
//    local pre-order, exactly the order the final numbering gives them.
// A host pass numbers the few large-range nodes in pre-order, placing each
// task's nodes as one contiguous block, and one kernel writes the tasks'
// nodes into the final arrays.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host/internal.h"

namespace sc {
namespace {

constexpr int kWarpBins = 32;    // bins per axis on the GPU (one per lane)
constexpr int kTaskMax = 2048;   // ranges up to this size are built by one warp
constexpr int kChunk = 4096;     // triangle positions per block in the large phase
constexpr int kBlock = 256;
constexpr int kTaskWarps = 4;    // warps (tasks) per block of the task kernel

#define CUDA_OK(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      fail(SC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

// Order-preserving integer images of floats and doubles, for atomic min/max.
__host__ __device__ inline uint32_t enc_f(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float dec_f(uint32_t u) {
  u = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
__host__ __device__ inline unsigned long long enc_d(double d) {
  unsigned long long u;
  std::memcpy(&u, &d, 8);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__host__ __device__ inline double dec_d(unsigned long long u) {
  u = (u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u;
  double d;
  std::memcpy(&d, &u, 8);
  return d;
}

// Encoded range statistics: box (min x3, max x3) and centroid bounds.
struct StatsO {
  uint32_t box[6];
  unsigned long long c[6];
};

// Bins of one range: counts and encoded boxes, [axis][bin].
struct BinsO {
  int cnt[3][kWarpBins];
  uint32_t box[3][kWarpBins][6];
};

// What the split of one range needs: its positions and centroid bounds.
struct SplitIn {
  int begin, end;
  double cmin[3], ext[3];
  int use[3];
};

struct Chunk {
  int range, begin, end;
};

// A node of a task's subtree, in the task's local pre-order.
struct LNode {
  int ch[2];   // leaf: first position; inner: local node id
  int cnt[2];  // leaf triangle count, 0 for an inner child
  float box[2][6];
  int depth;
};

struct Task {
  int begin, end, depth;
};

__device__ __forceinline__ double area_d(const float* b) {
  const double dx = __dsub_rn((double)b[3], (double)b[0]);
  const double dy = __dsub_rn((double)b[4], (double)b[1]);
  const double dz = __dsub_rn((double)b[5], (double)b[2]);
  return __dmul_rn(2.0, __dadd_rn(__dadd_rn(__dmul_rn(dx, dy), __dmul_rn(dy, dz)),
                                  __dmul_rn(dz, dx)));
}

__device__ __forceinline__ int bin_of(double c, double cmin, double ext, int nb) {
  int i = __double2int_rz(__dmul_rn(__dsub_rn(c, cmin), __ddiv_rn((double)nb, ext)));
  if (i > nb - 1) i = nb - 1;
  if (i < 0) i = 0;
  return i;
}

// A triangle index read from the order array; anything outside [0, n) is
// recorded as an internal error and skipped.
__device__ __forceinline__ bool tri_ok(int t, int n, int* err) {
  if ((unsigned)t < (unsigned)n) return true;
  atomicExch(err, 2);
  return false;
}

__global__ void prep_kernel(const float* __restrict__ tris, int64_t n, float* __restrict__ tb,
                            double* __restrict__ tc, int32_t* __restrict__ perm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* t = tris + 9 * i;
  for (int k = 0; k < 3; ++k) {
    const float lo = fminf(fminf(t[k], t[3 + k]), t[6 + k]);
    const float hi = fmaxf(fmaxf(t[k], t[3 + k]), t[6 + k]);
    tb[6 * i + k] = lo;
    tb[6 * i + 3 + k] = hi;
    tc[3 * i + k] = __dmul_rn(0.5, __dadd_rn((double)lo, (double)hi));
  }
  perm[i] = (int32_t)i;
}

__global__ void stats_init_kernel(StatsO* st, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < 3; ++k) {
    st[i].box[k] = enc_f(INFINITY);
    st[i].box[3 + k] = enc_f(-INFINITY);
    st[i].c[k] = enc_d(INFINITY);
    st[i].c[3 + k] = enc_d(-INFINITY);
  }
}

__global__ void bins_init_kernel(BinsO* bins, int n) {
  const int i = blockIdx.x;
  if (i >= n) return;
  for (int j = threadIdx.x; j < 3 * kWarpBins; j += blockDim.x) {
    const int k = j / kWarpBins, b = j % kWarpBins;
    bins[i].cnt[k][b] = 0;
    for (int q = 0; q < 3; ++q) {
      bins[i].box[k][b][q] = enc_f(INFINITY);
      bins[i].box[k][b][3 + q] = enc_f(-INFINITY);
    }
  }
}

// Box and centroid bounds of each chunk's triangles, merged into its range.
__global__ void stats_kernel(const Chunk* __restrict__ chunks, const int32_t* __restrict__ perm,
                             const float* __restrict__ tb, const double* __restrict__ tc,
                             StatsO* st, int n, int* err) {
  const Chunk ch = chunks[blockIdx.x];
  float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  double c[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  for (int i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) {
    const int t = perm[i];
    if (!tri_ok(t, n, err)) continue;
    for (int k = 0; k < 3; ++k) {
      b[k] = fminf(b[k], tb[6 * t + k]);
      b[3 + k] = fmaxf(b[3 + k], tb[6 * t + 3 + k]);
      const double ck = tc[3 * t + k];
      c[k] = ck < c[k] ? ck : c[k];
      c[3 + k] = ck > c[3 + k] ? ck : c[3 + k];
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    for (int k = 0; k < 3; ++k) {
      b[k] = fminf(b[k], __shfl_xor_sync(0xffffffffu, b[k], off));
      b[3 + k] = fmaxf(b[3 + k], __shfl_xor_sync(0xffffffffu, b[3 + k], off));
      const double lo = __shfl_xor_sync(0xffffffffu, c[k], off);
      const double hi = __shfl_xor_sync(0xffffffffu, c[3 + k], off);
      c[k] = lo < c[k] ? lo : c[k];
      c[3 + k] = hi > c[3 + k] ? hi : c[3 + k];
    }
  }
  if ((threadIdx.x & 31) == 0) {
    StatsO& s = st[ch.range];
    for (int k = 0; k < 3; ++k) {
      atomicMin(&s.box[k], enc_f(b[k]));
      atomicMax(&s.box[3 + k], enc_f(b[3 + k]));
      atomicMin(&s.c[k], enc_d(c[k]));
      atomicMax(&s.c[3 + k], enc_d(c[3 + k]));
    }
  }
}

// Adds triangle t to the bins of each used axis (shared or global memory).
__device__ __forceinline__ void bin_tri(BinsO& bins, const SplitIn& s, const float* tb,
                                        const double* tc, int t, int nb) {
  for (int k = 0; k < 3; ++k) {
    if (!s.use[k]) continue;
    const int bi = bin_of(tc[3 * t + k], s.cmin[k], s.ext[k], nb);
    atomicAdd(&bins.cnt[k][bi], 1);
    for (int q = 0; q < 3; ++q) {
      atomicMin(&bins.box[k][bi][q], enc_f(tb[6 * t + q]));
      atomicMax(&bins.box[k][bi][3 + q], enc_f(tb[6 * t + 3 + q]));
    }
  }
}

__global__ void bins_kernel(const Chunk* __restrict__ chunks, const SplitIn* __restrict__ sp,
                            const int32_t* __restrict__ perm, const float* __restrict__ tb,
                            const double* __restrict__ tc, BinsO* bins, int nb, int n,
                            int* err) {
  __shared__ BinsO sb;
  const Chunk ch = chunks[blockIdx.x];
  const SplitIn s = sp[ch.range];
  for (int j = threadIdx.x; j < 3 * kWarpBins; j += blockDim.x) {
    const int k = j / kWarpBins, b = j % kWarpBins;
    sb.cnt[k][b] = 0;
    for (int q = 0; q < 3; ++q) {
      sb.box[k][b][q] = enc_f(INFINITY);
      sb.box[k][b][3 + q] = enc_f(-INFINITY);
    }
  }
  __syncthreads();
  for (int i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) {
    const int t = perm[i];
    if (tri_ok(t, n, err)) bin_tri(sb, s, tb, tc, t, nb);
  }
  __syncthreads();
  BinsO& g = bins[ch.range];
  for (int j = threadIdx.x; j < 3 * kWarpBins; j += blockDim.x) {
    const int k = j / kWarpBins, b = j % kWarpBins;
    if (sb.cnt[k][b] == 0) continue;
    atomicAdd(&g.cnt[k][b], sb.cnt[k][b]);
    for (int q = 0; q < 3; ++q) {
      atomicMin(&g.box[k][b][q], sb.box[k][b][q]);
      atomicMax(&g.box[k][b][3 + q], sb.box[k][b][3 + q]);
    }
  }
}

// The cost sweep of one range by one warp, lane = bin: prefix (bins 0..p)
// and suffix (bins p+1..nb-1) counts and boxes by shuffles, the cost of
// every plane, and the lowest (cost, axis, plane).  Returns the axis (-1:
// no valid plane) and sets the plane.
__device__ int warp_sah(const BinsO& bins, const int* use, int nb, int lane, int& plane) {
  double best = INFINITY;
  int best_axis = -1;
  plane = -1;
  for (int k = 0; k < 3; ++k) {
    if (!use[k]) continue;
    int c = 0;
    float bx[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    if (lane < nb) {
      c = bins.cnt[k][lane];
      for (int q = 0; q < 6; ++q) bx[q] = dec_f(bins.box[k][lane][q]);
    }
    int lc = c, rc = c;
    float L[6], Rb[6];
    for (int q = 0; q < 6; ++q) L[q] = Rb[q] = bx[q];
    for (int off = 1; off < 32; off <<= 1) {
      const int tl = __shfl_up_sync(0xffffffffu, lc, off);
      const int tr = __shfl_down_sync(0xffffffffu, rc, off);
      float vl[6], vr[6];
      for (int q = 0; q < 6; ++q) {
        vl[q] = __shfl_up_sync(0xffffffffu, L[q], off);
        vr[q] = __shfl_down_sync(0xffffffffu, Rb[q], off);
      }
      if (lane >= off) {
        lc += tl;
        for (int q = 0; q < 3; ++q) {
          L[q] = fminf(L[q], vl[q]);
          L[3 + q] = fmaxf(L[3 + q], vl[3 + q]);
        }
      }
      if (lane + off < 32) {
        rc += tr;
        for (int q = 0; q < 3; ++q) {
          Rb[q] = fminf(Rb[q], vr[q]);
          Rb[3 + q] = fmaxf(Rb[3 + q], vr[3 + q]);
        }
      }
    }
    // right side of plane `lane` = suffix starting at bin lane + 1
    const int rcount = __shfl_down_sync(0xffffffffu, rc, 1);
    float R[6];
    for (int q = 0; q < 6; ++q) R[q] = __shfl_down_sync(0xffffffffu, Rb[q], 1);
    double cost = INFINITY;
    if (lane < nb - 1 && lc > 0 && rcount > 0)
      cost = __dadd_rn(__dmul_rn(area_d(L), (double)lc), __dmul_rn(area_d(R), (double)rcount));
    int pl = lane;
    for (int off = 16; off > 0; off >>= 1) {
      const double oc = __shfl_xor_sync(0xffffffffu, cost, off);
      const int op = __shfl_xor_sync(0xffffffffu, pl, off);
      if (oc < cost || (oc == cost && op < pl)) {
        cost = oc;
        pl = op;
      }
    }
    if (cost < best) {
      best = cost;
      best_axis = k;
      plane = pl;
    }
  }
  return best_axis;
}

__global__ void sah_kernel(const SplitIn* __restrict__ sp, const BinsO* __restrict__ bins,
                           int nranges, int nb, int2* __restrict__ split) {
  const int r = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= nranges) return;  // uniform across the warp
  int plane;
  const int axis = warp_sah(bins[r], sp[r].use, nb, lane, plane);
  if (lane == 0) split[r] = make_int2(axis, plane);
}

__device__ __forceinline__ bool goes_left(const SplitIn& s, int2 sl, const double* tc, int t,
                                          int nb) {
  return bin_of(tc[3 * t + sl.x], s.cmin[sl.x], s.ext[sl.x], nb) <= sl.y;
}

__device__ __forceinline__ int block_sum(int v, int* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  int s = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  __syncthreads();
  return s;
}

__global__ void count_kernel(const Chunk* __restrict__ chunks, const SplitIn* __restrict__ sp,
                             const int2* __restrict__ split, const int32_t* __restrict__ perm,
                             const double* __restrict__ tc, int nb, int* __restrict__ nleft,
                             int n, int* err) {
  __shared__ int red[32];
  const Chunk ch = chunks[blockIdx.x];
  const int2 sl = split[ch.range];
  int c = 0;
  if (sl.x >= 0) {
    const SplitIn s = sp[ch.range];
    for (int i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) {
      const int t = perm[i];
      if (tri_ok(t, n, err)) c += goes_left(s, sl, tc, t, nb);
    }
  }
  c = block_sum(c, red);
  if (threadIdx.x == 0) nleft[blockIdx.x] = c;
}

// Stable partition of each chunk into tmp: left triangles at the range's
// start plus the lefts of earlier chunks, rights after all of the range's
// lefts.  Thread j of the block owns positions [j*per, (j+1)*per) of the
// chunk, in order.
__global__ void scatter_kernel(const Chunk* __restrict__ chunks, const SplitIn* __restrict__ sp,
                               const int2* __restrict__ split, const int* __restrict__ loff,
                               const int* __restrict__ range_nl, const int32_t* __restrict__ perm,
                               const double* __restrict__ tc, int nb, int32_t* __restrict__ tmp,
                               int n, int* err) {
  __shared__ int wsum[32];
  const Chunk ch = chunks[blockIdx.x];
  const int2 sl = split[ch.range];
  if (sl.x < 0) return;  // half split: the order is kept
  const SplitIn s = sp[ch.range];
  const int per = (kChunk + kBlock - 1) / kBlock;
  const int p0 = ch.begin + threadIdx.x * per;
  const int p1 = min(p0 + per, ch.end);
  int nl = 0;
  for (int i = p0; i < p1; ++i) {
    const int t = perm[i];
    if (tri_ok(t, n, err)) nl += goes_left(s, sl, tc, t, nb);
  }
  // exclusive block scan of nl
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = nl;
  for (int off = 1; off < 32; off <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  int before = 0;
  for (int i = 0; i < w; ++i) before += wsum[i];
  const int lex = before + incl - nl;                       // lefts before this thread
  const int items_before = max(0, min(p0, ch.end) - ch.begin);
  int li = s.begin + loff[blockIdx.x] + lex;
  int ri = s.begin + range_nl[ch.range] + (ch.begin - s.begin - loff[blockIdx.x]) +
           (items_before - lex);
  for (int i = p0; i < p1; ++i) {
    const int t = perm[i];
    if (!tri_ok(t, n, err)) continue;
    const int dst = goes_left(s, sl, tc, t, nb) ? li++ : ri++;
    if (dst >= s.begin && dst < s.end) tmp[dst] = t;
    else atomicExch(err, 3);
  }
}

__global__ void copy_back_kernel(const Chunk* __restrict__ chunks, const int2* __restrict__ split,
                                 const int32_t* __restrict__ tmp, int32_t* __restrict__ perm) {
  const Chunk ch = chunks[blockIdx.x];
  if (split[ch.range].x < 0) return;
  for (int i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) perm[i] = tmp[i];
}

// One warp builds the subtree of one task range: ranges depth first, left
// before right, each one's statistics, then (if it holds more than
// max_leaf triangles) a node, its bins, the cost sweep and the stable
// partition.  Pending right ranges wait on a stack at the task's own
// positions (there are fewer than the task's triangles), and the task's
// local nodes (fewer than its triangles) sit at the same offsets.
__global__ void __launch_bounds__(32 * kTaskWarps)
    task_kernel(const Task* __restrict__ tasks, int ntasks, int32_t* __restrict__ perm,
                int32_t* __restrict__ tmp, const float* __restrict__ tb,
                const double* __restrict__ tc, int nb, int max_leaf, LNode* __restrict__ ln,
                int4* __restrict__ stack, int* __restrict__ task_nodes,
                int* __restrict__ task_depth, int ntri, int* __restrict__ err) {
  __shared__ BinsO sbins[kTaskWarps];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ti = blockIdx.x * kTaskWarps + wid;
  if (ti >= ntasks) return;  // uniform across the warp
  BinsO& bins = sbins[wid];
  const Task task = tasks[ti];
  const int base = task.begin, nt = task.end - task.begin;
  LNode* nodes = ln + base;
  int4* stk = stack + base;
  int sp = 0, nodes_made = 0, max_depth = task.depth, steps = 0;
  int4 cur = make_int4(task.begin, task.end, task.depth, -1);  // (begin, end, depth, parent*2+side)
  for (;;) {
    if (++steps > 2 * nt + 2) {  // cannot happen: every step splits or ends a range
      if (lane == 0) atomicExch(err, 1);
      break;
    }
    const int begin = cur.x, end = cur.y, depth = cur.z, n = end - begin;
    float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    double c[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int i = begin + lane; i < end; i += 32) {
      const int t = perm[i];
      if (!tri_ok(t, ntri, err)) continue;
      for (int k = 0; k < 3; ++k) {
        b[k] = fminf(b[k], tb[6 * t + k]);
        b[3 + k] = fmaxf(b[3 + k], tb[6 * t + 3 + k]);
        const double ck = tc[3 * t + k];
        c[k] = ck < c[k] ? ck : c[k];
        c[3 + k] = ck > c[3 + k] ? ck : c[3 + k];
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      for (int k = 0; k < 3; ++k) {
        b[k] = fminf(b[k], __shfl_xor_sync(0xffffffffu, b[k], off));
        b[3 + k] = fmaxf(b[3 + k], __shfl_xor_sync(0xffffffffu, b[3 + k], off));
        const double lo = __shfl_xor_sync(0xffffffffu, c[k], off);
        const double hi = __shfl_xor_sync(0xffffffffu, c[3 + k], off);
        c[k] = lo < c[k] ? lo : c[k];
        c[3 + k] = hi > c[3 + k] ? hi : c[3 + k];
      }
    }
    max_depth = max(max_depth, depth);
    const bool leaf = n <= max_leaf;
    // a task of nt triangles has at most nt - 1 nodes and nt - 1 pending
    // ranges; more means an internal error, recorded, and the task stops
    if (!leaf && (nodes_made >= nt - 1 || sp >= nt - 1 || n < 2)) {
      if (lane == 0) atomicExch(err, 4);
      break;
    }
    const int id = leaf ? -1 : nodes_made++;
    if (lane == 0) {
      if (cur.w >= 0) {
        LNode& p = nodes[cur.w >> 1];
        const int side = cur.w & 1;
        p.ch[side] = leaf ? begin : id;
        p.cnt[side] = leaf ? n : 0;
        for (int q = 0; q < 6; ++q) p.box[side][q] = b[q];
      }
      if (!leaf) nodes[id].depth = depth;
    }
    if (!leaf) {
      SplitIn s;
      s.begin = begin;
      s.end = end;
      for (int k = 0; k < 3; ++k) {
        s.cmin[k] = c[k];
        s.ext[k] = __dsub_rn(c[3 + k], c[k]);
        s.use[k] = s.ext[k] > 0.0;
      }
      for (int j = lane; j < 3 * kWarpBins; j += 32) {
        const int k = j / kWarpBins, bb = j % kWarpBins;
        bins.cnt[k][bb] = 0;
        for (int q = 0; q < 3; ++q) {
          bins.box[k][bb][q] = enc_f(INFINITY);
          bins.box[k][bb][3 + q] = enc_f(-INFINITY);
        }
      }
      __syncwarp();
      for (int i = begin + lane; i < end; i += 32) {
        const int t = perm[i];
        if (tri_ok(t, ntri, err)) bin_tri(bins, s, tb, tc, t, nb);
      }
      __syncwarp();
      int plane;
      const int axis = warp_sah(bins, s.use, nb, lane, plane);
      __syncwarp();
      int mid;
      if (axis < 0) {
        mid = begin + n / 2;
      } else {
        const int2 sl = make_int2(axis, plane);
        const unsigned lt = (1u << lane) - 1u;
        int nl = 0, nr = 0;
        for (int i0 = begin; i0 < end; i0 += 32) {
          const int i = i0 + lane;
          const bool valid = i < end;
          const int t = valid ? perm[i] : 0;
          const bool left = valid && tri_ok(t, ntri, err) && goes_left(s, sl, tc, t, nb);
          const unsigned bl = __ballot_sync(0xffffffffu, left);
          const unsigned br = __ballot_sync(0xffffffffu, valid && !left);
          __syncwarp();
          // every lane has read its position before any write; a left lands
          // at or before its own position, a right goes to tmp
          if (left) perm[begin + nl + __popc(bl & lt)] = t;
          else if (valid) tmp[begin + nr + __popc(br & lt)] = t;
          nl += __popc(bl);
          nr += __popc(br);
          __syncwarp();
        }
        for (int j = lane; j < nr; j += 32) perm[begin + nl + j] = tmp[begin + j];
        __syncwarp();
        mid = begin + nl;
      }
      if (lane == 0) stk[sp] = make_int4(mid, end, depth + 1, id * 2 + 1);
      __syncwarp();
      ++sp;
      cur = make_int4(begin, mid, depth + 1, id * 2);
      continue;
    }
    if (sp == 0) break;
    --sp;
    cur = stk[sp];
  }
  if (lane == 0) {
    task_nodes[ti] = nodes_made;
    task_depth[ti] = max_depth;
  }
}

// Writes each task's nodes at its place in the pre-order numbering.
__global__ void emit_kernel(const Task* __restrict__ tasks, const int* __restrict__ task_base,
                            const int* __restrict__ task_nodes, const LNode* __restrict__ ln,
                            int32_t* __restrict__ child, int32_t* __restrict__ count,
                            float* __restrict__ box, int32_t* __restrict__ ndepth) {
  const int ti = blockIdx.x;
  const int base = task_base[ti], cnt = task_nodes[ti];
  const LNode* nodes = ln + tasks[ti].begin;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const LNode& nd = nodes[j];
    const int64_t g = (int64_t)base + j;
    for (int s = 0; s < 2; ++s) {
      child[2 * g + s] = nd.cnt[s] > 0 ? nd.ch[s] : base + nd.ch[s];
      count[2 * g + s] = nd.cnt[s];
      for (int q = 0; q < 6; ++q) box[12 * g + 6 * s + q] = nd.box[s][q];
    }
    ndepth[g] = nd.depth;
  }
}

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

// A growable device array (per-level tables).  Growing waits for the
// stream first: kernels queued earlier may still read the old array.
template <class T>
struct DevVec {
  T* p = nullptr;
  size_t cap = 0;
  T* need(size_t n, cudaStream_t st) {
    if (n > cap) {
      CUDA_OK(cudaStreamSynchronize(st));
      if (p) cudaFree(p);
      p = nullptr;
      cap = std::max<size_t>(n, 2 * cap);
      CUDA_OK(cudaMalloc(&p, cap * sizeof(T)));
    }
    return p;
  }
  ~DevVec() {
    if (p) cudaFree(p);
  }
};

template <class T>
T* put(DevVec<T>& d, const std::vector<T>& v, cudaStream_t st) {
  T* p = d.need(v.size(), st);
  if (!v.empty()) CUDA_OK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return p;
}

// A range met in the large phase: its positions, depth, decoded statistics
// and what it became.
struct HRange {
  int begin, end, depth;
  float box[6];
  double cmin[3], cmax[3];
  int kind = 0;  // 0 leaf, 1 task, 2 large node
  int index = -1;  // task index or large-node index
};

struct HNode {
  int range;     // HRange of the node
  int ch[2];     // HRange of each child
};

}  // namespace

void build_bvh_gpu(Bvh& b, const float* tris, int64_t n, int max_leaf, int bins) {
  const double t0 = now_ms();
  if (bins > kWarpBins)
    fail(SC_ERR_UNSUPPORTED, "the GPU builder bins at most %d planes per axis (bins = %d)",
         kWarpBins, bins);
  b.ntri = n;
  b.tris.assign(tris, tris + 9 * n);
  b.perm.resize((size_t)n);
  b.child.clear();
  b.count.clear();
  b.box.clear();
  b.ndepth.clear();
  b.nn = 0;
  b.max_depth = 0;
  if (n == 0) {
    b.root_child = -1;
    b.root_count = 0;
    for (int k = 0; k < 3; ++k) {
      b.root_box[k] = INFINITY;
      b.root_box[3 + k] = -INFINITY;
    }
    b.ms_bvh = now_ms() - t0;
    return;
  }
  cudaStream_t st = nullptr;
  CUDA_OK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } guard{st};
  DevBufs d;
  float* d_tris = d.alloc<float>(9 * (size_t)n);
  float* tb = d.alloc<float>(6 * (size_t)n);
  double* tc = d.alloc<double>(3 * (size_t)n);
  int32_t* perm = d.alloc<int32_t>((size_t)n);
  int32_t* tmp = d.alloc<int32_t>((size_t)n);
  int* err = d.alloc<int>(1);
  CUDA_OK(cudaMemcpyAsync(d_tris, tris, 9 * (size_t)n * sizeof(float), cudaMemcpyHostToDevice, st));
  CUDA_OK(cudaMemsetAsync(err, 0, sizeof(int), st));
  prep_kernel<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(d_tris, n, tb, tc, perm);
  CUDA_OK(cudaGetLastError());

  DevVec<Chunk> d_chunks;
  DevVec<StatsO> d_stats;
  DevVec<SplitIn> d_sp;
  DevVec<BinsO> d_bins;
  DevVec<int2> d_split;
  DevVec<int> d_nleft, d_loff, d_rnl;
  std::vector<HRange> ranges;
  std::vector<HNode> big;
  std::vector<Task> tasks;
  std::vector<int> task_range;
  std::vector<Chunk> chunks;
  std::vector<StatsO> hstats;

  auto chunk_table = [&](const std::vector<int>& ids) {
    chunks.clear();
    for (int r = 0; r < (int)ids.size(); ++r) {
      const HRange& R = ranges[ids[r]];
      for (int p = R.begin; p < R.end; p += kChunk) chunks.push_back(Chunk{r, p, std::min(p + kChunk, R.end)});
    }
  };
  // Statistics of new ranges, then what each becomes.
  auto settle = [&](const std::vector<int>& ids, std::vector<int>& large) {
    large.clear();
    if (ids.empty()) return;
    chunk_table(ids);
    Chunk* dc = put(d_chunks, chunks, st);
    StatsO* ds = d_stats.need(ids.size(), st);
    stats_init_kernel<<<(unsigned)((ids.size() + 127) / 128), 128, 0, st>>>(ds, (int)ids.size());
    stats_kernel<<<(unsigned)chunks.size(), kBlock, 0, st>>>(dc, perm, tb, tc, ds, (int)n, err);
    CUDA_OK(cudaGetLastError());
    hstats.resize(ids.size());
    CUDA_OK(cudaMemcpyAsync(hstats.data(), ds, ids.size() * sizeof(StatsO), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaStreamSynchronize(st));
    for (size_t r = 0; r < ids.size(); ++r) {
      HRange& R = ranges[ids[r]];
      for (int k = 0; k < 6; ++k) R.box[k] = dec_f(hstats[r].box[k]);
      for (int k = 0; k < 3; ++k) {
        R.cmin[k] = dec_d(hstats[r].c[k]);
        R.cmax[k] = dec_d(hstats[r].c[3 + k]);
      }
      b.max_depth = std::max(b.max_depth, R.depth);
      const int cnt = R.end - R.begin;
      if (cnt <= max_leaf) {
        R.kind = 0;
      } else if (cnt <= kTaskMax) {
        R.kind = 1;
        R.index = (int)tasks.size();
        tasks.push_back(Task{R.begin, R.end, R.depth});
        task_range.push_back(ids[r]);
      } else {
        R.kind = 2;
        large.push_back(ids[r]);
      }
    }
  };

  ranges.push_back(HRange{0, (int)n, 0});
  std::vector<int> level{0}, large, next;
  settle(level, large);
  std::vector<SplitIn> sps;
  std::vector<int2> hsplit;
  std::vector<int> nleft, loff, rnl;
  while (!large.empty()) {
    // bins and the cost sweep of every large range of this level
    sps.resize(large.size());
    for (size_t r = 0; r < large.size(); ++r) {
      const HRange& R = ranges[large[r]];
      SplitIn& s = sps[r];
      s.begin = R.begin;
      s.end = R.end;
      for (int k = 0; k < 3; ++k) {
        s.cmin[k] = R.cmin[k];
        s.ext[k] = R.cmax[k] - R.cmin[k];
        s.use[k] = s.ext[k] > 0.0;
      }
    }
    const int nr = (int)large.size();
    chunk_table(large);
    const int nc = (int)chunks.size();
    Chunk* dc = put(d_chunks, chunks, st);
    SplitIn* dsp = put(d_sp, sps, st);
    BinsO* db = d_bins.need(nr, st);
    int2* dsl = d_split.need(nr, st);
    int* dnl = d_nleft.need(nc, st);
    bins_init_kernel<<<nr, 128, 0, st>>>(db, nr);
    bins_kernel<<<nc, kBlock, 0, st>>>(dc, dsp, perm, tb, tc, db, bins, (int)n, err);
    sah_kernel<<<(unsigned)((nr * 32 + 127) / 128), 128, 0, st>>>(dsp, db, nr, bins, dsl);
    count_kernel<<<nc, kBlock, 0, st>>>(dc, dsp, dsl, perm, tc, bins, dnl, (int)n, err);
    CUDA_OK(cudaGetLastError());
    hsplit.resize(nr);
    nleft.resize(nc);
    int herr = 0;
    CUDA_OK(cudaMemcpyAsync(hsplit.data(), dsl, nr * sizeof(int2), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(nleft.data(), dnl, nc * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaStreamSynchronize(st));
    if (herr) fail(SC_ERR_STATE, "GPU BVH builder: internal error %d", herr);
    // left offsets of each chunk within its range, and each range's lefts
    loff.resize(nc);
    rnl.assign(nr, 0);
    for (int c = 0; c < nc; ++c) {
      loff[c] = rnl[chunks[c].range];
      rnl[chunks[c].range] += nleft[c];
    }
    put(d_loff, loff, st);
    put(d_rnl, rnl, st);
    scatter_kernel<<<nc, kBlock, 0, st>>>(dc, dsp, dsl, d_loff.p, d_rnl.p, perm, tc, bins, tmp,
                                          (int)n, err);
    copy_back_kernel<<<nc, kBlock, 0, st>>>(dc, dsl, tmp, perm);
    CUDA_OK(cudaGetLastError());
    next.clear();
    for (int r = 0; r < nr; ++r) {
      const int id = large[r];
      const int begin = ranges[id].begin, end = ranges[id].end, depth = ranges[id].depth;
      const int mid = hsplit[r].x < 0 ? begin + (end - begin) / 2 : begin + rnl[r];
      if (mid <= begin || mid >= end) fail(SC_ERR_STATE, "GPU BVH builder: empty split side");
      ranges[id].index = (int)big.size();
      HNode nd;
      nd.range = id;
      nd.ch[0] = (int)ranges.size();
      ranges.push_back(HRange{begin, mid, depth + 1});
      nd.ch[1] = (int)ranges.size();
      ranges.push_back(HRange{mid, end, depth + 1});
      big.push_back(nd);
      next.push_back(nd.ch[0]);
      next.push_back(nd.ch[1]);
    }
    settle(next, large);
  }

  // every task's subtree, one warp each
  const int ntasks = (int)tasks.size();
  std::vector<int> tnodes(ntasks), tdepth(ntasks);
  LNode* ln = d.alloc<LNode>((size_t)n);
  int* d_tnodes = d.alloc<int>(ntasks);
  int* d_tdepth = d.alloc<int>(ntasks);
  Task* d_tasks = d.alloc<Task>(ntasks);
  if (ntasks > 0) {
    int4* stack = d.alloc<int4>((size_t)n);
    CUDA_OK(cudaMemcpyAsync(d_tasks, tasks.data(), ntasks * sizeof(Task), cudaMemcpyHostToDevice, st));
    task_kernel<<<(ntasks + kTaskWarps - 1) / kTaskWarps, 32 * kTaskWarps, 0, st>>>(
        d_tasks, ntasks, perm, tmp, tb, tc, bins, max_leaf, ln, stack, d_tnodes, d_tdepth, (int)n,
        err);
    CUDA_OK(cudaGetLastError());
    CUDA_OK(cudaMemcpyAsync(tnodes.data(), d_tnodes, ntasks * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(tdepth.data(), d_tdepth, ntasks * sizeof(int), cudaMemcpyDeviceToHost, st));
    int herr = 0;
    CUDA_OK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaStreamSynchronize(st));
    if (herr) fail(SC_ERR_STATE, "GPU BVH builder: internal error %d", herr);
    for (int t = 0; t < ntasks; ++t) b.max_depth = std::max(b.max_depth, tdepth[t]);
  }

  // pre-order numbering: large nodes one by one, each task as one block
  const HRange& root = ranges[0];
  std::memcpy(b.root_box, root.box, sizeof(b.root_box));
  if (root.kind == 0) {
    b.root_child = root.begin;
    b.root_count = root.end - root.begin;
  } else {
    b.root_child = 0;
    b.root_count = 0;
  }
  int64_t nn = (int64_t)big.size();
  for (int t = 0; t < ntasks; ++t) nn += tnodes[t];
  if (nn >= ((int64_t)1 << 31)) fail(SC_ERR_UNSUPPORTED, "too many BVH nodes");
  b.nn = nn;
  b.child.assign(2 * (size_t)nn, 0);
  b.count.assign(2 * (size_t)nn, 0);
  b.box.assign(12 * (size_t)nn, 0.0f);
  b.ndepth.assign((size_t)nn, 0);
  std::vector<int> task_base(ntasks, 0);
  std::vector<int> big_id(big.size(), -1);
  if (root.kind != 0) {
    struct Item {
      int range;
      int64_t parent_slot;
    };
    std::vector<Item> stk{{0, -1}};
    int64_t nxt = 0;
    while (!stk.empty()) {
      const Item it = stk.back();
      stk.pop_back();
      const HRange& R = ranges[it.range];
      const int64_t id = nxt;
      if (R.kind == 1) {
        task_base[R.index] = (int)id;
        nxt += tnodes[R.index];
      } else {
        nxt += 1;
        big_id[R.index] = (int)id;
      }
      if (it.parent_slot >= 0) b.child[it.parent_slot] = (int32_t)id;
      if (R.kind != 2) continue;
      const HNode& nd = big[R.index];
      b.ndepth[id] = R.depth;
      for (int c = 1; c >= 0; --c) {
        const HRange& C = ranges[nd.ch[c]];
        std::memcpy(&b.box[12 * id + 6 * c], C.box, sizeof(C.box));
        if (C.kind == 0) {
          b.child[2 * id + c] = C.begin;
          b.count[2 * id + c] = C.end - C.begin;
        } else {
          b.count[2 * id + c] = 0;
          stk.push_back(Item{nd.ch[c], 2 * id + c});
        }
      }
    }
    if (nxt != nn) fail(SC_ERR_STATE, "GPU BVH builder: node numbering mismatch");
  }
  if (ntasks > 0) {
    int32_t* d_child = d.alloc<int32_t>(2 * (size_t)nn);
    int32_t* d_count = d.alloc<int32_t>(2 * (size_t)nn);
    float* d_box = d.alloc<float>(12 * (size_t)nn);
    int32_t* d_nd = d.alloc<int32_t>((size_t)nn);
    int* d_base = d.alloc<int>(ntasks);
    CUDA_OK(cudaMemcpyAsync(d_base, task_base.data(), ntasks * sizeof(int), cudaMemcpyHostToDevice, st));
    emit_kernel<<<ntasks, 128, 0, st>>>(d_tasks, d_base, d_tnodes, ln, d_child, d_count, d_box, d_nd);
    CUDA_OK(cudaGetLastError());
    // task nodes from the device; the large nodes (set above) are kept
    std::vector<int32_t> c2(2 * (size_t)nn), n2(2 * (size_t)nn), dd((size_t)nn);
    std::vector<float> bx(12 * (size_t)nn);
    CUDA_OK(cudaMemcpyAsync(c2.data(), d_child, c2.size() * 4, cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(n2.data(), d_count, n2.size() * 4, cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(bx.data(), d_box, bx.size() * 4, cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(dd.data(), d_nd, dd.size() * 4, cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(b.perm.data(), perm, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaStreamSynchronize(st));
    for (int t = 0; t < ntasks; ++t) {
      const int64_t lo = task_base[t], hi = lo + tnodes[t];
      std::copy(c2.begin() + 2 * lo, c2.begin() + 2 * hi, b.child.begin() + 2 * lo);
      std::copy(n2.begin() + 2 * lo, n2.begin() + 2 * hi, b.count.begin() + 2 * lo);
      std::copy(bx.begin() + 12 * lo, bx.begin() + 12 * hi, b.box.begin() + 12 * lo);
      std::copy(dd.begin() + lo, dd.begin() + hi, b.ndepth.begin() + lo);
    }
  } else {
    CUDA_OK(cudaMemcpyAsync(b.perm.data(), perm, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaStreamSynchronize(st));
  }
  int herr = 0;
  CUDA_OK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) fail(SC_ERR_STATE, "GPU BVH builder: internal error %d", herr);
  b.ms_bvh = now_ms() - t0;
}

}  // namespace sc
