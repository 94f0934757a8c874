// trace_kernel.cuh — persistent-warp BVH2 traversal with subspace culling
// for sm_103a (templates; instantiated by trace_r*.cu).
//
// One thread traces one ray at a time; each warp takes batches of 32 ray
// indices from a global counter (one atomicAdd per batch, broadcast by
// shuffle) until the rays run out.  Per visited inner node the thread loads
// the 64-byte child-pair record with four 128-bit read-only loads, runs the
// two slab tests, and for every child the ray's box segment hits it runs the
// culling test of Sec. 3.1.2: the clipped segment ends p0 = o + tn*d and
// p1 = o + tf*d are quantised to cells (Alg. 1), the ray mask for the
// (begin, end) cell pair is looked up, and the child survives iff the AND
// with its object mask is non-zero (Alg. 4).  Traversal order: if both
// children survive the nearer (smaller tn) is visited next and the other is
// pushed with its tn; a popped entry with tn > current closest t is dropped.
//
// Every floating-point test op is written with explicit round-to-nearest
// intrinsics (__fadd_rn, __fmul_rn, ...), so no multiply-add contraction can
// change a decision: the op sequence is the canonical one a CPU reference
// performs in IEEE float.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sct {

constexpr uint32_t kLeaf = 0x80000000u;
constexpr float kRobust = 1.00000047683715820f;  // 1 + 4 * 2^-23 >= 1 + 2 gamma_3
constexpr int kStack = 64;

enum { ST_OK = 0, ST_STACK = 1, ST_BAD_NODE = 2 };

struct __align__(16) Hit {
  float t;
  int id;
  float u, v;
};

struct Params {
  const float4* nodes;
  int node_f4;              // node stride in float4 units
  const float4* tris;       // 3 float4 per triangle
  const uint4* lut;         // full ray-mask table (mask stride bytes per entry)
  const uint2* pair;        // factored 2-D table, R^4 x 64 bits
  const uint4* clut;        // compression LUT
  const float4* rays;       // 2 float4 per ray
  Hit* hits;
  uint2* counts;            // or nullptr
  unsigned* work;           // [0] ray counter, [1] status
  long long n;
  long long num_nodes;      // inner nodes in the image
  long long num_tris;
  uint32_t root_slot;
  int has_root;
};

// A slot may be followed only if it stays inside the image and, for an
// inner node, has a larger index than its parent (pre-order numbering): this
// bounds every ray's work even if the image were corrupted.
__device__ __forceinline__ bool slot_ok(uint32_t s, long long parent, const Params& p) {
  if (s & kLeaf) {
    const long long first = (long long)(s & 0x0FFFFFFFu);
    const long long cnt = (long long)((s >> 28) & 7u) + 1;
    return first + cnt <= p.num_tris;
  }
  return (long long)s > parent && (long long)s < p.num_nodes;
}

__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }
__device__ __forceinline__ uint4 ldg4u(const uint4* p) { return __ldg(p); }

// Alg. 1 on one axis, with a clamp at 0 and a floor on the extent.
template <int R>
__device__ __forceinline__ int cell_of(float p, float lo, float hi) {
  const float ext = __fsub_rn(hi, lo);
  const float s = __fdiv_rn((float)R, fmaxf(ext, 1e-30f));
  float q = __fmul_rn(__fsub_rn(p, lo), s);
  q = fminf(fmaxf(q, -1.0f), (float)R);
  int i = (int)floorf(q);
  i = i < 0 ? 0 : i;
  return i > R - 1 ? R - 1 : i;
}

// Object mask words of child c of a node record (uncompressed layout).
template <int R>
struct MaskTraits {
  static constexpr int kStrideBytes = (R == 4) ? 8 : (R == 6 ? 32 : 64);
  static constexpr int kQuads = kStrideBytes / 16;  // 0 for R = 4
  static constexpr int kR3 = R * R * R;
};

// AND of two masks in global memory (16-B aligned, zero padded) != 0.
template <int R>
__device__ __forceinline__ bool masks_overlap(const void* a, const void* b) {
  if constexpr (R == 4) {
    uint2 x = __ldg(reinterpret_cast<const uint2*>(a));
    uint2 y = __ldg(reinterpret_cast<const uint2*>(b));
    return ((x.x & y.x) | (x.y & y.y)) != 0u;
  } else {
    unsigned acc = 0;
#pragma unroll
    for (int q = 0; q < MaskTraits<R>::kQuads; ++q) {
      uint4 x = ldg4u(reinterpret_cast<const uint4*>(a) + q);
      uint4 y = ldg4u(reinterpret_cast<const uint4*>(b) + q);
      acc |= (x.x & y.x) | (x.y & y.y) | (x.z & y.z) | (x.w & y.w);
    }
    return acc != 0u;
  }
}

// Ray-mask table staged in shared memory in factored form: one 2-D sweep
// table P over (begin, end) cells of a pair of axes (Helly's theorem makes
// the 3-D mask the AND of the (x,y), (y,z) and (x,z) tables), plus two
// 2^R-entry expansion tables that turn an R-bit set of rows / columns into
// an R^2-bit slice.
template <int R>
struct SmemLut {
  unsigned long long P[R * R * R * R];
  unsigned long long rows[1 << R];  // y-set -> R^2 bits (whole rows)
  unsigned long long cols[1 << R];  // x-set -> R^2 bits (one per row)
};

template <int R>
__device__ void stage_lut(SmemLut<R>& s, const uint2* pair) {
  for (int i = threadIdx.x; i < R * R * R * R; i += blockDim.x) {
    uint2 v = pair[i];
    s.P[i] = (unsigned long long)v.x | ((unsigned long long)v.y << 32);
  }
  for (int m = threadIdx.x; m < (1 << R); m += blockDim.x) {
    unsigned long long r = 0, c = 0;
    for (int k = 0; k < R; ++k) {
      if ((m >> k) & 1) r |= ((1ULL << R) - 1ULL) << (R * k);
      c |= (unsigned long long)m << (R * k);
    }
    s.rows[m] = r;
    s.cols[m] = c;
  }
}

// R^2-bit slice z of a dense R^3-bit mask held in W words.
template <int R>
__device__ __forceinline__ unsigned long long mask_slice(const uint32_t* w, int z) {
  constexpr int S = R * R;
  const int bit = S * z;
  const int wi = bit >> 5, sh = bit & 31;
  unsigned long long lo = w[wi];
  unsigned long long hi = (wi + 1 < (R * R * R + 31) / 32) ? w[wi + 1] : 0u;
  unsigned long long hh = (wi + 2 < (R * R * R + 31) / 32) ? w[wi + 2] : 0u;
  unsigned long long v = (lo | (hi << 32)) >> sh;
  if (sh + S > 64) v |= hh << (64 - sh);
  if constexpr (S == 64) {
    return v;
  } else {
    return v & ((1ULL << S) - 1ULL);
  }
}

template <int R>
__device__ __forceinline__ bool overlap_factored(const SmemLut<R>& s, const int* cb,
                                                 const int* ce, const uint32_t* obj) {
  auto pidx = [](int ba, int bb, int ea, int eb) { return ((ba * R + bb) * R + ea) * R + eb; };
  const unsigned long long pxy = s.P[pidx(cb[0], cb[1], ce[0], ce[1])];
  const unsigned long long pyz = s.P[pidx(cb[1], cb[2], ce[1], ce[2])];
  const unsigned long long pxz = s.P[pidx(cb[0], cb[2], ce[0], ce[2])];
  const int z0 = min(cb[2], ce[2]), z1 = max(cb[2], ce[2]);
  constexpr unsigned long long m = (1ULL << R) - 1ULL;
  for (int z = z0; z <= z1; ++z) {
    unsigned long long ray = pxy & s.rows[(pyz >> (R * z)) & m] & s.cols[(pxz >> (R * z)) & m];
    if (ray & mask_slice<R>(obj, z)) return true;
  }
  return false;
}

// LUT variants: 0 = full table in global memory (one 8/32/64-byte entry per
// lookup, served by L1/L2), 1 = factored tables in shared memory.
template <int R, int CULL, int MODE, int LUTV>
__global__ void __launch_bounds__(128) trace_kernel(Params p) {
  constexpr int R3 = (R > 0) ? R * R * R : 1;
  constexpr int W = (R3 + 31) / 32;
  constexpr int MB = (R > 0) ? MaskTraits<(R > 0 ? R : 4)>::kStrideBytes : 8;
  __shared__ SmemLut<(R > 0 ? R : 4)> slut;
  if constexpr (CULL != 0 && LUTV == 1) {
    stage_lut<R>(slut, p.pair);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(&p.work[0], 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((long long)base >= p.n) break;
    const long long rid = (long long)base + lane;
    if (rid < p.n) {
      const float4 ra = __ldg(&p.rays[2 * rid]);
      const float4 rb = __ldg(&p.rays[2 * rid + 1]);
      const float ox = ra.x, oy = ra.y, oz = ra.z, tmin = ra.w;
      const float dx = rb.x, dy = rb.y, dz = rb.z;
      const float ix = __fdiv_rn(1.0f, dx), iy = __fdiv_rn(1.0f, dy), iz = __fdiv_rn(1.0f, dz);
      float tcur = rb.w;
      float ht = __int_as_float(0x7f800000), hu = 0.0f, hv = 0.0f;
      int hid = -1;
      unsigned ntest = 0, ttest = 0;
      uint2 stack[kStack];
      int sp = 0;
      uint32_t cur = p.root_slot;
      bool have = p.has_root != 0;
      bool done = false;
      while (!done) {
        if (have) {
          if (cur & kLeaf) {
            const int first = (int)(cur & 0x0FFFFFFFu);
            const int cnt = (int)((cur >> 28) & 7u) + 1;
            for (int i = 0; i < cnt; ++i) {
              const float4* tp = p.tris + 3 * (long long)(first + i);
              const float4 A = ldg4(tp), E1 = ldg4(tp + 1), E2 = ldg4(tp + 2);
              ++ttest;
              // Moeller-Trumbore, canonical op order
              const float px = __fsub_rn(__fmul_rn(dy, E2.z), __fmul_rn(dz, E2.y));
              const float py = __fsub_rn(__fmul_rn(dz, E2.x), __fmul_rn(dx, E2.z));
              const float pz = __fsub_rn(__fmul_rn(dx, E2.y), __fmul_rn(dy, E2.x));
              const float det = __fadd_rn(__fadd_rn(__fmul_rn(E1.x, px), __fmul_rn(E1.y, py)),
                                          __fmul_rn(E1.z, pz));
              if (det == 0.0f) continue;
              const float inv = __fdiv_rn(1.0f, det);
              const float sx = __fsub_rn(ox, A.x), sy = __fsub_rn(oy, A.y), sz = __fsub_rn(oz, A.z);
              const float u = __fmul_rn(
                  __fadd_rn(__fadd_rn(__fmul_rn(sx, px), __fmul_rn(sy, py)), __fmul_rn(sz, pz)), inv);
              if (u < 0.0f || u > 1.0f) continue;
              const float qx = __fsub_rn(__fmul_rn(sy, E1.z), __fmul_rn(sz, E1.y));
              const float qy = __fsub_rn(__fmul_rn(sz, E1.x), __fmul_rn(sx, E1.z));
              const float qz = __fsub_rn(__fmul_rn(sx, E1.y), __fmul_rn(sy, E1.x));
              const float v = __fmul_rn(
                  __fadd_rn(__fadd_rn(__fmul_rn(dx, qx), __fmul_rn(dy, qy)), __fmul_rn(dz, qz)), inv);
              if (v < 0.0f || __fadd_rn(u, v) > 1.0f) continue;
              const float t = __fmul_rn(
                  __fadd_rn(__fadd_rn(__fmul_rn(E2.x, qx), __fmul_rn(E2.y, qy)), __fmul_rn(E2.z, qz)),
                  inv);
              if (!(t > tmin && t < tcur)) continue;
              ht = t;
              hu = u;
              hv = v;
              hid = __float_as_int(A.w);
              if (MODE == 1) {
                done = true;
                break;
              }
              tcur = t;
            }
            have = false;
            continue;
          }
          const float4* nd = p.nodes + (long long)cur * p.node_f4;
          const float4 f0 = ldg4(nd), f1 = ldg4(nd + 1), f2 = ldg4(nd + 2);
          const uint4 f3 = ldg4u(reinterpret_cast<const uint4*>(nd + 3));
          ntest += 2;
          const float lo0[3] = {f0.x, f0.y, f0.z}, hi0[3] = {f0.w, f1.x, f1.y};
          const float lo1[3] = {f1.z, f1.w, f2.x}, hi1[3] = {f2.y, f2.z, f2.w};
          const float o[3] = {ox, oy, oz}, inv[3] = {ix, iy, iz};
          float tn[2], tf[2];
          bool hit[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const float* lo = c ? lo1 : lo0;
            const float* hi = c ? hi1 : hi0;
            float a0[3], a1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              a0[k] = __fmul_rn(__fsub_rn(lo[k], o[k]), inv[k]);
              a1[k] = __fmul_rn(__fsub_rn(hi[k], o[k]), inv[k]);
            }
            tn[c] = fmaxf(fmaxf(fminf(a0[0], a1[0]), fminf(a0[1], a1[1])),
                          fmaxf(fminf(a0[2], a1[2]), tmin));
            tf[c] = fminf(fminf(fmaxf(a0[0], a1[0]), fmaxf(a0[1], a1[1])),
                          fminf(fmaxf(a0[2], a1[2]), tcur));
            hit[c] = tn[c] <= __fmul_rn(tf[c], kRobust);
          }
          if constexpr (CULL != 0) {
            const float d[3] = {dx, dy, dz};
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              if (!hit[c]) continue;
              const float* lo = c ? lo1 : lo0;
              const float* hi = c ? hi1 : hi0;
              int cb[3], ce[3];
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                const float p0 = __fadd_rn(o[k], __fmul_rn(tn[c], d[k]));
                const float p1 = __fadd_rn(o[k], __fmul_rn(tf[c], d[k]));
                cb[k] = cell_of<R>(p0, lo[k], hi[k]);
                ce[k] = cell_of<R>(p1, lo[k], hi[k]);
              }
              const uint8_t* obj;
              if constexpr (CULL == 1) {
                obj = reinterpret_cast<const uint8_t*>(nd + 4) + c * MB;
              } else {
                const unsigned idx = (c ? f3.w : f3.z) & 0xFFu;
                obj = reinterpret_cast<const uint8_t*>(p.clut) + idx * MB;
              }
              if constexpr (LUTV == 0) {
                const int beg = cb[0] + R * cb[1] + R * R * cb[2];
                const int end = ce[0] + R * ce[1] + R * R * ce[2];
                const uint8_t* rm = reinterpret_cast<const uint8_t*>(p.lut) + (size_t)(beg * R3 + end) * MB;
                hit[c] = masks_overlap<R>(rm, obj);
              } else {
                uint32_t w[W + 1];
                if constexpr (R == 4) {
                  const uint2 q = __ldg(reinterpret_cast<const uint2*>(obj));
                  w[0] = q.x;
                  w[1] = q.y;
                } else {
#pragma unroll
                  for (int i = 0; i < MB / 16; ++i) {
                    const uint4 q = ldg4u(reinterpret_cast<const uint4*>(obj) + i);
                    if (4 * i + 0 < W) w[4 * i + 0] = q.x;
                    if (4 * i + 1 < W) w[4 * i + 1] = q.y;
                    if (4 * i + 2 < W) w[4 * i + 2] = q.z;
                    if (4 * i + 3 < W) w[4 * i + 3] = q.w;
                  }
                }
                w[W] = 0u;
                hit[c] = overlap_factored<R>(slut, cb, ce, w);
              }
            }
          }
          const uint32_t s0 = f3.x, s1 = f3.y;
          if ((hit[0] && !slot_ok(s0, (long long)cur, p)) ||
              (hit[1] && !slot_ok(s1, (long long)cur, p))) {
            atomicOr(&p.work[1], (unsigned)ST_BAD_NODE);
            done = true;
            continue;
          }
          if (hit[0] && hit[1]) {
            const int nr = tn[1] < tn[0] ? 1 : 0;
            if (sp < kStack) {
              stack[sp] = make_uint2(nr ? s0 : s1, __float_as_uint(nr ? tn[0] : tn[1]));
              ++sp;
            } else {
              atomicOr(&p.work[1], (unsigned)ST_STACK);
              done = true;
            }
            cur = nr ? s1 : s0;
          } else if (hit[0]) {
            cur = s0;
          } else if (hit[1]) {
            cur = s1;
          } else {
            have = false;
          }
          continue;
        }
        while (sp > 0) {
          --sp;
          if (__uint_as_float(stack[sp].y) > tcur) continue;
          cur = stack[sp].x;
          have = true;
          break;
        }
        if (!have) done = true;
      }
      Hit h;
      h.t = ht;
      h.id = hid;
      h.u = hu;
      h.v = hv;
      reinterpret_cast<float4*>(p.hits)[rid] =
          make_float4(h.t, __int_as_float(h.id), h.u, h.v);
      if (p.counts) p.counts[rid] = make_uint2(ntest, ttest);
    }
  }
}

// Launch entry for one variant.
typedef void (*KernelFn)(Params);

}  // namespace sct
