// trace_kernel.cuh — persistent-warp BVH2 traversal with subspace culling
// for sm_103a (templates; instantiated by trace_r*.cu / trace_plain.cu).
//
// Work distribution: each warp keeps 32 rays in flight.  Whenever enough of
// its lanes have finished (ballot), the warp takes that many new ray indices
// from a global counter with one atomicAdd and hands them to the idle lanes,
// so lanes do not wait for the slowest ray of a batch.
//
// Per step a lane either visits one inner node or tests the triangles of one
// leaf.  An inner-node visit loads the child-pair record with 128-bit
// read-only loads, runs the two slab tests and, for every child whose box the
// ray segment hits, the culling test of Sec. 3.1.2: the clipped segment ends
// p0 = o + tn*d and p1 = o + tf*d are quantised to cells (Alg. 1), the ray
// mask of the (begin, end) cell pair is looked up, and the child survives
// iff the AND with its object mask is non-zero (Alg. 4).  Order: if both
// children survive, the one with the smaller entry distance is visited next
// and the other is pushed with its entry distance; a popped entry is dropped
// unless it would still pass the widened slab test (tn <= tcur * kRobust).
//
// Every floating-point test op is an explicit round-to-nearest intrinsic
// (__fadd_rn, __fmul_rn, ...), so no multiply-add contraction can change a
// decision: the op sequence is the canonical one a CPU reference performs in
// IEEE float, which makes hits and per-ray test counts reproducible.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sct {

constexpr uint32_t kLeaf = 0x80000000u;
constexpr uint32_t kMetaFull = 0x100u;   // child mask is all ones: the test cannot cull
constexpr float kRobust = 1.00000047683715820f;  // 1 + 4 * 2^-23 >= 1 + 2 gamma_3
constexpr int kStack = 64;
constexpr int kBlock = 128;
// Leaf triangles tested per traversal step; a longer leaf continues in the
// next steps.  One per step measured fastest for both traversals: lanes at
// leaves then keep pace with lanes at inner nodes.
constexpr int kTrisPerStep = 1;

enum { ST_OK = 0, ST_STACK = 1, ST_BAD_NODE = 2 };

struct Params {
  const float4* nodes;
  int node_f4;              // node stride in float4 units
  int mask_off_f4;          // first object mask inside a record (float4 units)
  const float4* tris;       // 3 float4 per triangle
  const uint4* lut;         // full ray-mask table (mask-stride bytes per entry)
  const uint2* pair;        // factored 2-D table, R^4 x 64 bits
  const uint4* clut;        // compression LUT
  const uint32_t* bits;     // compressed: [R^6][8] words, bit j of row = ray mask AND LUT entry j
  const uint4* lut2;        // R_ray = 2R table ((2R)^6 rows, mask-stride bytes), or nullptr
  const float4* rays;       // 2 float4 per ray
  float4* hits;             // {t, id bits, u, v}
  uint2* counts;            // or nullptr
  unsigned* work;           // ray counter(s) / control words
  unsigned* status;         // device status word (ST_* bits)
  long long n;
  long long num_nodes;      // inner nodes in the image
  long long num_tris;
  uint32_t root_slot;
  int has_root;
  int refill;               // refill when at least this many lanes are idle
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

// 32 bytes from a 32-byte aligned read-only address with one 256-bit load
// (sm_100 family).  Used for the 32- and 64-byte object masks and ray-mask
// rows: node records are whole 32-byte sectors with their masks on 32-byte
// offsets, and every image region starts on a 256-byte boundary.
__device__ __forceinline__ void ldg8u(const void* p, uint4& a, uint4& b) {
  asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
      : "l"(p));
}

// The same 256-bit load without allocating the line in L1 (NA), for rows of
// the ray-mask tables: random 32- or 64-byte rows of a 1.49 MB (96 MB at
// R_ray = 2R) table that few other lanes read again, which would otherwise
// evict node records that neighbouring rays fetch next.
template <bool NA>
__device__ __forceinline__ void ldg8u_row(const void* p, uint4& a, uint4& b) {
  if constexpr (NA) {
    asm("ld.global.nc.L1::no_allocate.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
        : "l"(p));
  } else {
    ldg8u(p, a, b);
  }
}

template <int R>
struct MaskTraits {
  static constexpr int kStrideBytes = (R == 4) ? 8 : (R == 6 ? 32 : 64);
  static constexpr int kQuads = kStrideBytes / 16;  // 0 for R = 4
  static constexpr int kWords = (R * R * R + 31) / 32;
};

// Kernel options (template bit field OPT).  None changes which nodes are
// visited; OPT_FUSED changes the rounding of the Alg. 1 cell coordinate and
// has its own oracle mode.
enum : int {
  OPT_FUSED = 1,  // Alg. 1 coordinate by one fused multiply-add in t (not the paper's order)
  OPT_PAIR = 2,   // the lookups of both children are in flight before either is used
  OPT_SPEC = 4,   // the nearer slab-passing child's record is fetched before the
                  // culling results arrive (and every next record at the end of a step)
  OPT_TOS = 8,    // the top stack entry is kept in registers
  OPT_SORT = 16,  // waves: each bounce queue is sorted by direction octant and
                  // origin cell before its wave is traced
  OPT_LAZY = 64,  // the per-child scales are loaded only when a child needs a test
  OPT_SSTACK = 128, // the top kRing stack entries in shared memory (blocks of kBlock)
  OPT_TL1 = 256,  // full-table rows and uncompressed object masks allocated in L1
                  // like other loads (by default they bypass L1 allocation)
  OPT_OCC9 = 1024,  // waves: 9 resident blocks of 128 threads per SM (56 registers)
                    // instead of 8 (64 registers)
  OPT_OCC10 = 2048, // waves: 10 resident blocks of 128 threads per SM (48 registers)
  OPT_HSLOT = 4096, // the accepted hit's u, v and triangle id kept in a per-thread
                    // shared-memory slot instead of three registers
  OPT_DEFER = 32, // compressed, bit table: a child's culling lookup is issued
                  // when the child is visited, beside its own fetch (the
                  // cells still come from the parent's slab test)
};

constexpr uint32_t kNoTest = 0xFFFFFFFFu;

// Rows of the full ray-mask table (R = 6, 8) and of the R_ray = 2R table,
// and the uncompressed object masks of the node records, skip L1
// allocation unless OPT_TL1 is set: both are fetched only for a tested
// child, while the records' boxes are what neighbouring rays fetch next.
template <int OPT>
constexpr bool kRowNA = (OPT & OPT_TL1) == 0;

// floor(q) clamped to [0, R-1]: the saturating float-to-unsigned conversion
// (cvt.rmi, negatives and NaN to 0) and a min.
template <int R>
__device__ __forceinline__ int cell_of_q(float q) {
  return (int)min(__float2uint_rd(q), (unsigned)(R - 1));
}

// Alg. 1 cell coordinates (before the floor) of the segment ends at tn and
// tf on one axis of a box with lower bound lo and scale s = R / extent.  As
// written: p = o + t d (product, then sum), then (p - lo) * s.  OPT_FUSED:
// s (o - lo) + t (s d) as one fused multiply-add.
template <int OPT>
__device__ __forceinline__ void cell_coords(float o, float d, float lo, float s, float tn,
                                            float tf, float& q0, float& q1) {
  if constexpr ((OPT & OPT_FUSED) != 0) {
    const float a = __fmul_rn(__fsub_rn(o, lo), s);
    const float b = __fmul_rn(d, s);
    q0 = __fmaf_rn(tn, b, a);
    q1 = __fmaf_rn(tf, b, a);
  } else {
    const float p0 = __fadd_rn(o, __fmul_rn(tn, d));
    const float p1 = __fadd_rn(o, __fmul_rn(tf, d));
    q0 = __fmul_rn(__fsub_rn(p0, lo), s);
    q1 = __fmul_rn(__fsub_rn(p1, lo), s);
  }
}

// Two FP32 lanes in one 64-bit register pair, and the sm_100-family packed
// operations on them (add / sub / mul .rn.f32x2): each lane is rounded to
// nearest exactly as the scalar __fadd_rn / __fsub_rn / __fmul_rn, so the
// packed forms below give the same bits as the scalar ones.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pk2(float a, float b) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void up2(f2x r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  f2x r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
  f2x r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
  f2x r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

// Alg. 1 cell coordinates of both segment ends on all three axes: x and y
// as packed pairs, z scalar (the same operations, lane by lane, as
// cell_coords); the fused option stays scalar.
template <int OPT>
__device__ __forceinline__ void cell_coords3(const float* o, const float* d, const float* lo,
                                             const float* sk, float tn, float tf, float* q0,
                                             float* q1) {
  if constexpr ((OPT & OPT_FUSED) != 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) cell_coords<OPT>(o[k], d[k], lo[k], sk[k], tn, tf, q0[k], q1[k]);
  } else {
    const f2x oxy = pk2(o[0], o[1]), dxy = pk2(d[0], d[1]);
    const f2x lxy = pk2(lo[0], lo[1]), sxy = pk2(sk[0], sk[1]);
    const f2x a = mul2(sub2(add2(oxy, mul2(pk2(tn, tn), dxy)), lxy), sxy);
    const f2x b = mul2(sub2(add2(oxy, mul2(pk2(tf, tf), dxy)), lxy), sxy);
    up2(a, q0[0], q0[1]);
    up2(b, q1[0], q1[1]);
    cell_coords<OPT>(o[2], d[2], lo[2], sk[2], tn, tf, q0[2], q1[2]);
  }
}

// Slab tests of the two children of a binary record (f0..f2 in the layout
// {lo0.xy, hi0.xy} {lo1.xy, hi1.xy} {lo0.z, hi0.z, lo1.z, hi1.z}): entry
// and exit distances clipped to [tmin, tcur], x and y as packed pairs.
// tn = max(max(near_x, near_y), max(near_z, tmin)), tf = min(min(far_x,
// far_y), min(far_z, tcur)); hit iff tn <= tf * kRobust.
__device__ __forceinline__ void slab2(const float4 f0, const float4 f1, const float4 f2,
                                      float ox, float oy, float oz, float ix, float iy, float iz,
                                      float tmin, float tcur, float* tn, float* tf, bool* hit) {
  const f2x oxy = pk2(ox, oy), ixy = pk2(ix, iy);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const float4 f = c ? f1 : f0;
    const float loz = c ? f2.z : f2.x, hiz = c ? f2.w : f2.y;
    float a0x, a0y, a1x, a1y;
    up2(mul2(sub2(pk2(f.x, f.y), oxy), ixy), a0x, a0y);
    up2(mul2(sub2(pk2(f.z, f.w), oxy), ixy), a1x, a1y);
    const float a0z = __fmul_rn(__fsub_rn(loz, oz), iz);
    const float a1z = __fmul_rn(__fsub_rn(hiz, oz), iz);
    tn[c] = fmaxf(fmaxf(fminf(a0x, a1x), fminf(a0y, a1y)), fmaxf(fminf(a0z, a1z), tmin));
    tf[c] = fminf(fminf(fmaxf(a0x, a1x), fmaxf(a0y, a1y)), fminf(fmaxf(a0z, a1z), tcur));
    hit[c] = tn[c] <= __fmul_rn(tf[c], kRobust);
  }
}

template <int R>
__device__ __forceinline__ float scale_of(float lo, float hi) {
  return __fdiv_rn((float)R, fmaxf(__fsub_rn(hi, lo), 1e-30f));
}

// AND of two masks in global memory (aligned, zero padded) != 0.  ROW_NA /
// OBJ_NA: the first (a ray-mask table row) / second (an object mask) is
// loaded without L1 allocation.
template <int R, bool ROW_NA = false, bool OBJ_NA = false>
__device__ __forceinline__ bool masks_overlap(const void* a, const void* b) {
  if constexpr (R == 4) {
    const uint2 x = __ldg(reinterpret_cast<const uint2*>(a));
    const uint2 y = __ldg(reinterpret_cast<const uint2*>(b));
    return ((x.x & y.x) | (x.y & y.y)) != 0u;
  } else {
    // masks of 32 / 64 bytes at 32-byte aligned offsets: 256-bit loads
    unsigned acc = 0;
#pragma unroll
    for (int q = 0; q < MaskTraits<R>::kQuads; q += 2) {
      uint4 x0, x1, y0, y1;
      ldg8u_row<ROW_NA>(reinterpret_cast<const uint4*>(a) + q, x0, x1);
      ldg8u_row<OBJ_NA>(reinterpret_cast<const uint4*>(b) + q, y0, y1);
      acc |= (x0.x & y0.x) | (x0.y & y0.y) | (x0.z & y0.z) | (x0.w & y0.w) | (x1.x & y1.x) |
             (x1.y & y1.y) | (x1.z & y1.z) | (x1.w & y1.w);
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

// R = 4 only: the whole ray-mask table (4,096 entries of 64 bits, 32 KB) and
// the compression LUT (256 x 64 bits) fit in shared memory, so a culling
// test needs no global-memory lookup on the step's critical path.
struct SmemFull4 {
  uint2 lut[4096];
  uint2 clut[256];
};

__device__ __forceinline__ void stage_full4(SmemFull4& s, const uint4* lut, const uint4* clut) {
  const uint2* l = reinterpret_cast<const uint2*>(lut);
  for (int i = threadIdx.x; i < 4096; i += blockDim.x) s.lut[i] = l[i];
  if (clut) {
    const uint2* c = reinterpret_cast<const uint2*>(clut);
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s.clut[i] = c[i];
  }
}

template <int R>
__device__ __forceinline__ void stage_lut(SmemLut<R>& s, const uint2* pair) {
  for (int i = threadIdx.x; i < R * R * R * R; i += blockDim.x) {
    const uint2 v = pair[i];
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

// Shared-memory tables of each lookup variant (nothing for the global ones).
template <int R, int LUTV>
struct SharedTables {
  int unused;
};
template <int R>
struct SharedTables<R, 1> {
  SmemLut<R> f;
};
template <>
struct SharedTables<4, 3> {
  SmemFull4 full;
};

// The two 2^R-entry expansion tables of SmemLut as read-only device data
// (for the factored test read through L1, lookup variant 5).
template <int R>
struct ExpandTables {
  unsigned long long rows[1 << R];
  unsigned long long cols[1 << R];
};

template <int R>
constexpr ExpandTables<R> make_expand() {
  ExpandTables<R> e{};
  for (int m = 0; m < (1 << R); ++m) {
    unsigned long long r = 0, c = 0;
    for (int k = 0; k < R; ++k) {
      if ((m >> k) & 1) r |= ((1ULL << R) - 1ULL) << (R * k);
      c |= (unsigned long long)m << (R * k);
    }
    e.rows[m] = r;
    e.cols[m] = c;
  }
  return e;
}

__device__ const ExpandTables<6> kExpand6 = make_expand<6>();

// R^2-bit slice z of a dense R^3-bit mask held in W (+1 zero) words.
template <int R>
__device__ __forceinline__ unsigned long long mask_slice(const uint32_t* w, int z) {
  constexpr int S = R * R;
  constexpr int W = MaskTraits<R>::kWords;
  const int bit = S * z;
  const int wi = bit >> 5, sh = bit & 31;
  const unsigned long long lo = w[wi];
  const unsigned long long hi = (wi + 1 < W) ? w[wi + 1] : 0u;
  unsigned long long v = (lo | (hi << 32)) >> sh;
  if (sh + S > 64) {
    const unsigned long long hh = (wi + 2 < W) ? w[wi + 2] : 0u;
    v |= hh << (64 - sh);
  }
  if constexpr (S == 64) {
    return v;
  } else {
    return v & ((1ULL << S) - 1ULL);
  }
}

// The factored test (Helly: the ray mask of slice z is the (x,y) table's
// R^2 bits restricted to the rows of the (y,z) table's set for z and the
// columns of the (x,z) table's set for z), slice by slice over the z range
// of the segment.  FROM_L1: the pair table and the expansion tables are
// read from global memory through L1 instead of from shared memory.
template <int R, bool FROM_L1 = false>
__device__ __forceinline__ bool overlap_factored(const SmemLut<R>* s, const uint2* gpair,
                                                 const int* cb, const int* ce,
                                                 const uint8_t* objp) {
  constexpr int W = MaskTraits<R>::kWords;
  uint32_t w[W + 1];
  if constexpr (R == 4) {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(objp));
    w[0] = q.x;
    w[1] = q.y;
  } else {
#pragma unroll
    for (int i = 0; i < MaskTraits<R>::kQuads; ++i) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(objp) + i);
      if (4 * i + 0 < W) w[4 * i + 0] = q.x;
      if (4 * i + 1 < W) w[4 * i + 1] = q.y;
      if (4 * i + 2 < W) w[4 * i + 2] = q.z;
      if (4 * i + 3 < W) w[4 * i + 3] = q.w;
    }
  }
  w[W] = 0u;
  auto pidx = [](int ba, int bb, int ea, int eb) { return ((ba * R + bb) * R + ea) * R + eb; };
  auto pget = [&](int i) -> unsigned long long {
    if constexpr (FROM_L1) {
      const uint2 v = __ldg(gpair + i);
      return (unsigned long long)v.x | ((unsigned long long)v.y << 32);
    } else {
      return s->P[i];
    }
  };
  const unsigned long long pxy = pget(pidx(cb[0], cb[1], ce[0], ce[1]));
  const unsigned long long pyz = pget(pidx(cb[1], cb[2], ce[1], ce[2]));
  const unsigned long long pxz = pget(pidx(cb[0], cb[2], ce[0], ce[2]));
  const int z0 = min(cb[2], ce[2]), z1 = max(cb[2], ce[2]);
  constexpr unsigned long long m = (1ULL << R) - 1ULL;
  for (int z = z0; z <= z1; ++z) {
    unsigned long long rsel, csel;
    if constexpr (FROM_L1) {
      static_assert(R == 6, "the L1 expansion tables are built for R = 6");
      rsel = __ldg(&kExpand6.rows[(pyz >> (R * z)) & m]);
      csel = __ldg(&kExpand6.cols[(pxz >> (R * z)) & m]);
    } else {
      rsel = s->rows[(pyz >> (R * z)) & m];
      csel = s->cols[(pxz >> (R * z)) & m];
    }
    if (pxy & rsel & csel & mask_slice<R>(w, z)) return true;
  }
  return false;
}

// Moeller-Trumbore, canonical op order.  Returns true and t, u, v on accept.
__device__ __forceinline__ bool tri_test(const float4 A, const float4 E1, const float4 E2,
                                         float ox, float oy, float oz, float dx, float dy,
                                         float dz, float tmin, float tcur, float& t, float& u,
                                         float& v) {
  const float px = __fsub_rn(__fmul_rn(dy, E2.z), __fmul_rn(dz, E2.y));
  const float py = __fsub_rn(__fmul_rn(dz, E2.x), __fmul_rn(dx, E2.z));
  const float pz = __fsub_rn(__fmul_rn(dx, E2.y), __fmul_rn(dy, E2.x));
  const float det =
      __fadd_rn(__fadd_rn(__fmul_rn(E1.x, px), __fmul_rn(E1.y, py)), __fmul_rn(E1.z, pz));
  if (det == 0.0f) return false;
  const float inv = __fdiv_rn(1.0f, det);
  const float sx = __fsub_rn(ox, A.x), sy = __fsub_rn(oy, A.y), sz = __fsub_rn(oz, A.z);
  u = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(sx, px), __fmul_rn(sy, py)), __fmul_rn(sz, pz)),
                inv);
  if (u < 0.0f || u > 1.0f) return false;
  const float qx = __fsub_rn(__fmul_rn(sy, E1.z), __fmul_rn(sz, E1.y));
  const float qy = __fsub_rn(__fmul_rn(sz, E1.x), __fmul_rn(sx, E1.z));
  const float qz = __fsub_rn(__fmul_rn(sx, E1.y), __fmul_rn(sy, E1.x));
  v = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, qx), __fmul_rn(dy, qy)), __fmul_rn(dz, qz)),
                inv);
  if (v < 0.0f || __fadd_rn(u, v) > 1.0f) return false;
  t = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(E2.x, qx), __fmul_rn(E2.y, qy)), __fmul_rn(E2.z, qz)),
                inv);
  return t > tmin && t < tcur;
}

template <int R, int LUTV>
__device__ __forceinline__ void stage_tables(SharedTables<R, LUTV>& sh, const Params& p) {
  if constexpr (LUTV == 1) {
    stage_lut<R>(sh.f, p.pair);
  } else if constexpr (LUTV == 3) {
    stage_full4(sh.full, p.lut, p.clut);
  }
}

// Record of one inner node as loaded: boxes, slots and meta words, and with
// stored scales the two float4 after them.
struct Rec {
  float4 f0, f1, f2, f3, f4, f5;
};

// A record is fetched with 128-bit loads: 256-bit loads of the records
// measured slower on the compressed 12.1M hair (23.4-23.9 against
// 23.2-23.5 ms per wave launch).
template <bool SCALED>
__device__ __forceinline__ void load_rec(const Params& p, uint32_t node, Rec& r) {
  const float4* nd = p.nodes + (long long)node * p.node_f4;
  r.f0 = __ldg(nd);
  r.f1 = __ldg(nd + 1);
  r.f2 = __ldg(nd + 2);
  r.f3 = __ldg(nd + 3);
  if constexpr (SCALED) {
    r.f4 = __ldg(nd + 4);
    r.f5 = __ldg(nd + 5);
  }
}

struct RayState {
  float ox, oy, oz, dx, dy, dz, ix, iy, iz, tmin, tcur;
  float ht, hu, hv;
  int hid;
  int hpos;   // leaf position of the accepted triangle (for bounce normals)
  unsigned ntest, ttest;
  int sp;
  uint32_t cur;
  bool have;  // `cur` is the next slot to visit (else pop)
  bool pre;   // OPT_SPEC: nx holds the record of `cur` (loaded or in flight)
  Rec nx;     // OPT_SPEC: prefetched record (its first four float4)
  uint2 top;  // OPT_TOS: the top stack entry (the array holds the ones below)
  uint32_t ctest;  // OPT_DEFER: pending test of `cur`: bit-table word index << 5 | bit, or kNoTest
};

// OPT_HSLOT: the u, v and triangle id of each thread's accepted hit live in
// shared memory (written at each accept, a few times per ray; read once when
// the ray finishes), which frees three registers.  Blocks of up to kMaxBlock
// threads.
constexpr int kMaxBlock = 256;
__device__ __forceinline__ float4* hit_slot() {
  __shared__ float4 slots[kMaxBlock];
  return slots + threadIdx.x;
}

// An accepted triangle at leaf position pos (A: its first float4, whose w is
// the id).
template <int OPT>
__device__ __forceinline__ void record_accept(RayState& s, float t, float u, float v,
                                              const float4 A, int pos) {
  s.ht = t;
  s.hpos = pos;
  if constexpr ((OPT & OPT_HSLOT) != 0) {
    *hit_slot() = make_float4(u, v, A.w, 0.0f);
  } else {
    s.hu = u;
    s.hv = v;
    s.hid = __float_as_int(A.w);
  }
}

__device__ __forceinline__ void ray_init(RayState& s, const float4 ra, const float4 rb,
                                         const Params& p) {
  s.ox = ra.x; s.oy = ra.y; s.oz = ra.z; s.tmin = ra.w;
  s.dx = rb.x; s.dy = rb.y; s.dz = rb.z; s.tcur = rb.w;
  s.ix = __fdiv_rn(1.0f, s.dx);
  s.iy = __fdiv_rn(1.0f, s.dy);
  s.iz = __fdiv_rn(1.0f, s.dz);
  s.ht = __int_as_float(0x7f800000);
  s.hu = 0.0f;
  s.hv = 0.0f;
  s.hid = -1;
  s.hpos = -1;
  s.ntest = 0;
  s.ttest = 0;
  s.sp = 0;
  s.cur = p.root_slot;
  s.have = p.has_root != 0;
  s.pre = false;
  s.ctest = kNoTest;
}

// The hit record {t, id bits, u, v} of a finished ray; {inf, -1, 0, 0} for
// a miss.
template <int OPT>
__device__ __forceinline__ float4 hit_record(const RayState& s) {
  if constexpr ((OPT & OPT_HSLOT) != 0) {
    if (s.hpos < 0) return make_float4(s.ht, __int_as_float(-1), 0.0f, 0.0f);
    const float4 h = *hit_slot();
    return make_float4(s.ht, h.z, h.x, h.y);
  } else {
    return make_float4(s.ht, __int_as_float(s.hid), s.hu, s.hv);
  }
}

// Culling test of one child from its record data: Alg. 1 cells of the
// segment [tn, tf] in the child's grid (lo, scales), the ray-mask lookup and
// the AND with the object mask `obj` (uncompressed) or LUT entry `meta`.
template <int R, int CULL, int LUTV, int OPT = 0>
__device__ __forceinline__ bool cull_test(const Params& p, const SharedTables<R, LUTV>& sh,
                                          const uint8_t* obj, unsigned meta, const float* lo,
                                          const float* sk, const float* o, const float* d,
                                          float tn, float tf) {
  constexpr int R3 = R * R * R;
  constexpr int MB = MaskTraits<R>::kStrideBytes;
  int cb[3], ce[3];
  if constexpr (LUTV == 4) {
    // R_ray = 2R (Sec. 4.2): cells of the 2R grid, twice the R-grid
    // coordinate (doubling is exact), one row per (begin, end) pair
    constexpr int R2 = 2 * R;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float q0, q1;
      cell_coords<OPT>(o[k], d[k], lo[k], sk[k], tn, tf, q0, q1);
      cb[k] = cell_of_q<R2>(__fmul_rn(2.0f, q0));
      ce[k] = cell_of_q<R2>(__fmul_rn(2.0f, q1));
    }
    const int beg2 = cb[0] + R2 * cb[1] + R2 * R2 * cb[2];
    const int end2 = ce[0] + R2 * ce[1] + R2 * R2 * ce[2];
    const uint8_t* rm =
        reinterpret_cast<const uint8_t*>(p.lut2) + ((size_t)beg2 * (R2 * R2 * R2) + end2) * MB;
    return masks_overlap<R, kRowNA<OPT>, kRowNA<OPT>>(rm, obj);
  }
  {
    float q0[3], q1[3];
    cell_coords3<OPT>(o, d, lo, sk, tn, tf, q0, q1);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cb[k] = cell_of_q<R>(q0[k]);
      ce[k] = cell_of_q<R>(q1[k]);
    }
  }
  const int beg = cb[0] + R * cb[1] + R * R * cb[2];
  const int end = ce[0] + R * ce[1] + R * R * ce[2];
  if constexpr (LUTV == 3) {
    const uint2 rm = sh.full.lut[beg * R3 + end];
    uint2 om;
    if constexpr (CULL == 1) {
      om = __ldg(reinterpret_cast<const uint2*>(obj));
    } else {
      om = sh.full.clut[meta & 0xFFu];
    }
    return ((rm.x & om.x) | (rm.y & om.y)) != 0u;
  } else if constexpr (CULL == 2 && LUTV == 2) {
    const unsigned j = meta & 0xFFu;
    const uint32_t word = __ldg(p.bits + (size_t)(beg * R3 + end) * 8 + (j >> 5));
    return (word >> (j & 31u)) & 1u;
  } else {
    if constexpr (CULL == 2) obj = reinterpret_cast<const uint8_t*>(p.clut) + (meta & 0xFFu) * MB;
    if constexpr (LUTV == 1) {
      return overlap_factored<R>(&sh.f, p.pair, cb, ce, obj);
    } else if constexpr (LUTV == 5) {
      return overlap_factored<R, true>(nullptr, p.pair, cb, ce, obj);
    } else {
      const uint8_t* rm = reinterpret_cast<const uint8_t*>(p.lut) + (size_t)(beg * R3 + end) * MB;
      return masks_overlap<R, kRowNA<OPT>, CULL == 1 && kRowNA<OPT>>(rm, obj);
    }
  }
}

// Stack push / pop.  OPT_TOS keeps the top entry in a register and the
// entries below it in the array, so a pop takes the register and refills it
// with a load whose latency hides behind the next node's work.
// OPT_SSTACK: a ring of the kRing top entries per thread in shared memory
// (entry k of thread t at ring[k * kBlock + t], conflict-free); entries
// further down live in the local array.  A push that overwrites a ring slot
// first moves its entry (kRing below the new top) to the array; a pop
// refills the freed slot from the array.
constexpr int kRing = 8;

__device__ __forceinline__ uint2* ring_array() {
  __shared__ uint2 ring[kBlock * kRing];
  return ring + threadIdx.x;
}

template <int STACK, int OPT>
__device__ __forceinline__ bool stack_push(RayState& s, uint2* stack, uint2 e) {
  if (s.sp >= STACK) return false;
  if constexpr ((OPT & OPT_SSTACK) != 0) {
    uint2* ring = ring_array();
    const int k = s.sp & (kRing - 1);
    if (s.sp >= kRing) stack[s.sp - kRing] = ring[k * kBlock];
    ring[k * kBlock] = e;
  } else if constexpr ((OPT & OPT_TOS) != 0) {
    if (s.sp > 0) stack[s.sp - 1] = s.top;
    s.top = e;
  } else {
    stack[s.sp] = e;
  }
  ++s.sp;
  return true;
}

template <int OPT>
__device__ __forceinline__ uint2 stack_pop(RayState& s, uint2* stack) {
  uint2 e;
  --s.sp;
  if constexpr ((OPT & OPT_SSTACK) != 0) {
    uint2* ring = ring_array();
    const int k = s.sp & (kRing - 1);
    e = ring[k * kBlock];
    if (s.sp >= kRing) ring[k * kBlock] = stack[s.sp - kRing];
  } else if constexpr ((OPT & OPT_TOS) != 0) {
    e = s.top;
    if (s.sp > 0) s.top = stack[s.sp - 1];
  } else {
    e = stack[s.sp];
  }
  return e;
}

// Begin and end cells (x + R y + R^2 z) of the clipped segment (Alg. 1).
template <int R, int OPT>
__device__ __forceinline__ int2 cell_pair(const float* o, const float* d, const float* lo,
                                          const float* sk, float tn, float tf) {
  float q0[3], q1[3];
  cell_coords3<OPT>(o, d, lo, sk, tn, tf, q0, q1);
  int cb[3], ce[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    cb[k] = cell_of_q<R>(q0[k]);
    ce[k] = cell_of_q<R>(q1[k]);
  }
  return make_int2(cb[0] + R * cb[1] + R * R * cb[2], ce[0] + R * ce[1] + R * R * ce[2]);
}

// A culling test split in two, so that the loads of several tests can be in
// flight together: lookup_issue computes the cells and issues the loads of
// the ray-mask row (or bit-table word) and object mask; lookup_result ANDs
// them.  Full table in global memory (LUTV 0, R <= 6) and bit table (LUTV 2).
template <int R, int CULL, int LUTV>
struct Lookup {
  static constexpr int kQ = MaskTraits<R>::kQuads;
  uint4 row[kQ > 0 ? kQ : 1], obj[kQ > 0 ? kQ : 1];
  uint2 row2, obj2;  // R = 4
  uint32_t word;     // bit table
  unsigned bit;
};

template <int R, int CULL, int LUTV, int OPT>
__device__ __forceinline__ void lookup_issue(const Params& p, Lookup<R, CULL, LUTV>& L,
                                             const uint8_t* obj, unsigned meta, const float* lo,
                                             const float* sk, const float* o, const float* d,
                                             float tn, float tf) {
  constexpr int R3 = R * R * R;
  constexpr int MB = MaskTraits<R>::kStrideBytes;
  const int2 be = cell_pair<R, OPT>(o, d, lo, sk, tn, tf);
  const size_t row = (size_t)(be.x * R3 + be.y);
  if constexpr (LUTV == 2) {
    const unsigned j = meta & 0xFFu;
    L.word = __ldg(p.bits + row * 8 + (j >> 5));
    L.bit = j & 31u;
  } else {
    if constexpr (CULL == 2) obj = reinterpret_cast<const uint8_t*>(p.clut) + (meta & 0xFFu) * MB;
    const uint8_t* rm = reinterpret_cast<const uint8_t*>(p.lut) + row * MB;
    if constexpr (R == 4) {
      L.row2 = __ldg(reinterpret_cast<const uint2*>(rm));
      L.obj2 = __ldg(reinterpret_cast<const uint2*>(obj));
    } else {
#pragma unroll
      for (int q = 0; q < Lookup<R, CULL, LUTV>::kQ; ++q) {
        L.row[q] = __ldg(reinterpret_cast<const uint4*>(rm) + q);
        L.obj[q] = __ldg(reinterpret_cast<const uint4*>(obj) + q);
      }
    }
  }
}

template <int R, int CULL, int LUTV>
__device__ __forceinline__ bool lookup_result(const Lookup<R, CULL, LUTV>& L) {
  if constexpr (LUTV == 2) {
    return (L.word >> L.bit) & 1u;
  } else if constexpr (R == 4) {
    return ((L.row2.x & L.obj2.x) | (L.row2.y & L.obj2.y)) != 0u;
  } else {
    unsigned acc = 0;
#pragma unroll
    for (int q = 0; q < Lookup<R, CULL, LUTV>::kQ; ++q)
      acc |= (L.row[q].x & L.obj[q].x) | (L.row[q].y & L.obj[q].y) |
             (L.row[q].z & L.obj[q].z) | (L.row[q].w & L.obj[q].w);
    return acc != 0u;
  }
}

// Pops the next entry that would still pass the widened slab test
// (tn <= tcur * kRobust: a child is kept or dropped alike whether it is
// reached directly or through the stack).  True when the stack is empty.
template <int OPT>
__device__ __forceinline__ bool pop_next(RayState& s, uint2* stack, uint32_t* tstack) {
  while (s.sp > 0) {
    const uint2 e = stack_pop<OPT>(s, stack);
    if (__uint_as_float(e.y) > __fmul_rn(s.tcur, kRobust)) continue;
    s.cur = e.x;
    if constexpr ((OPT & OPT_DEFER) != 0) s.ctest = tstack[s.sp];
    s.have = true;
    return false;
  }
  return true;
}

// The inner-node visit of the deferred variant (compressed masks, bit
// table, stored scales): the two slab tests, and for each slab-passing
// child that needs a culling test its bit-table word index and bit (from
// Alg. 1 cells of its clipped segment, computed now), carried with the
// child to its visit; then the near-first order of trace_step.  Node tests
// are counted here, so a child culled at its visit is counted as never
// visited.  Returns true when the ray has finished.
template <int R, int STACK>
__device__ __forceinline__ bool trace_inner_deferred(const Params& p, RayState& s, uint2* stack,
                                                     uint32_t* tstack, const float4* nd,
                                                     const Rec& rc) {
  constexpr int R3 = R * R * R;
  const float4 f0 = rc.f0, f1 = rc.f1, f2 = rc.f2;
  const uint32_t s0 = __float_as_uint(rc.f3.x), s1 = __float_as_uint(rc.f3.y);
  const uint32_t m0 = __float_as_uint(rc.f3.z), m1 = __float_as_uint(rc.f3.w);
  s.ntest += 2;
  const float lo0[3] = {f0.x, f0.y, f2.x}, lo1[3] = {f1.x, f1.y, f2.z};
  const float o[3] = {s.ox, s.oy, s.oz};
  const float d[3] = {s.dx, s.dy, s.dz};
  const float sc0[3] = {rc.f4.x, rc.f4.y, rc.f5.x}, sc1[3] = {rc.f4.z, rc.f4.w, rc.f5.y};
  float tn[2], tf[2];
  bool hit[2];
  slab2(f0, f1, f2, s.ox, s.oy, s.oz, s.ix, s.iy, s.iz, s.tmin, s.tcur, tn, tf, hit);
  uint32_t code[2] = {kNoTest, kNoTest};
  if (hit[0] && !(m0 & kMetaFull)) {
    const int2 be = cell_pair<R, 0>(o, d, lo0, sc0, tn[0], tf[0]);
    const uint32_t j = m0 & 0xFFu;
    code[0] = ((uint32_t)(be.x * R3 + be.y) * 8u + (j >> 5)) << 5 | (j & 31u);
  }
  if (hit[1] && !(m1 & kMetaFull)) {
    const int2 be = cell_pair<R, 0>(o, d, lo1, sc1, tn[1], tf[1]);
    const uint32_t j = m1 & 0xFFu;
    code[1] = ((uint32_t)(be.x * R3 + be.y) * 8u + (j >> 5)) << 5 | (j & 31u);
  }
  if ((hit[0] && !slot_ok(s0, (long long)s.cur, p)) ||
      (hit[1] && !slot_ok(s1, (long long)s.cur, p))) {
    atomicOr(p.status, (unsigned)ST_BAD_NODE);
    return true;
  }
  if (hit[0] && hit[1]) {
    const int nr = tn[1] < tn[0] ? 1 : 0;
    if (s.sp >= STACK) {
      atomicOr(p.status, (unsigned)ST_STACK);
      return true;
    }
    stack[s.sp] = make_uint2(nr ? s0 : s1, __float_as_uint(nr ? tn[0] : tn[1]));
    tstack[s.sp] = nr ? code[0] : code[1];
    ++s.sp;
    s.cur = nr ? s1 : s0;
    s.ctest = nr ? code[1] : code[0];
    return false;
  }
  if (hit[0] || hit[1]) {
    s.cur = hit[0] ? s0 : s1;
    s.ctest = hit[0] ? code[0] : code[1];
    return false;
  }
  s.have = false;
  return pop_next<OPT_DEFER>(s, stack, tstack);
}

// One traversal step of one ray: either the triangles of one leaf or one
// inner node, then a pop if nothing is left to visit.  Returns true when the
// ray has finished (or was stopped by a recorded device error).  The OPT
// bits change only when loads are issued and where the top stack entry
// lives, never which nodes are visited.
template <int R, int CULL, int MODE, int LUTV, int SCALES, int STACK = kStack, int OPT = 0>
__device__ __forceinline__ bool trace_step(const Params& p, RayState& s, uint2* stack,
                                           const SharedTables<(R > 0 ? R : 4), LUTV>& sh,
                                           uint32_t* tstack = nullptr) {
  constexpr int RR = (R > 0 ? R : 4);
  constexpr int MB = MaskTraits<RR>::kStrideBytes;
  constexpr bool kScaled = CULL != 0 && SCALES != 0;
  constexpr bool kSpec = (OPT & OPT_SPEC) != 0;
  constexpr bool kSplit = CULL != 0 && (LUTV == 2 || (LUTV == 0 && RR <= 6)) &&
                          (OPT & (OPT_PAIR | OPT_SPEC)) != 0;
  constexpr bool kDefer = (OPT & OPT_DEFER) != 0;
  static_assert((OPT & OPT_SSTACK) == 0 || (OPT & (OPT_TOS | OPT_DEFER)) == 0,
                "one stack placement at a time");
  static_assert(!kDefer || (CULL == 2 && LUTV == 2 && kTrisPerStep == 1 &&
                            (OPT & (OPT_PAIR | OPT_SPEC | OPT_TOS)) == 0),
                "the deferred test is built for the compressed bit table alone");
  bool done = false;
  if constexpr (kDefer) {
    // the pending culling test of the slot about to be visited: its
    // bit-table word is requested beside the slot's own fetch; a culled
    // slot is left without a test count, as if its parent had culled it
    if (s.have && s.ctest != kNoTest) {
      const uint32_t code = s.ctest;
      s.ctest = kNoTest;
      const uint32_t word = __ldg(p.bits + (code >> 5));
      if (s.cur & kLeaf) {
        const float4* tp = p.tris + 3 * (long long)(s.cur & 0x0FFFFFFFu);
        const float4 A = __ldg(tp), E1 = __ldg(tp + 1), E2 = __ldg(tp + 2);
        if (!((word >> (code & 31u)) & 1u)) {
          s.have = false;
        } else {
          const int first = (int)(s.cur & 0x0FFFFFFFu);
          const int left = (int)((s.cur >> 28) & 7u) + 1;
          ++s.ttest;
          float t, u, v;
          if (tri_test(A, E1, E2, s.ox, s.oy, s.oz, s.dx, s.dy, s.dz, s.tmin, s.tcur, t, u, v)) {
            record_accept<OPT>(s, t, u, v, A, first);
            if (MODE == 1) return true;
            s.tcur = t;
          }
          if (left > 1) {
            s.cur = kLeaf | ((uint32_t)(left - 2) << 28) | (uint32_t)(first + 1);
            return false;
          }
          s.have = false;
        }
      } else {
        const float4* nd = p.nodes + (long long)s.cur * p.node_f4;
        Rec rc;
        load_rec<true>(p, s.cur, rc);
        if (!((word >> (code & 31u)) & 1u)) {
          s.have = false;
        } else {
          return trace_inner_deferred<RR, STACK>(p, s, stack, tstack, nd, rc);
        }
      }
    }
  }
  if (s.have) {
    if (s.cur & kLeaf) {
      const int first = (int)(s.cur & 0x0FFFFFFFu);
      const int left = (int)((s.cur >> 28) & 7u) + 1;
      // at most kTrisPerStep triangles per step; the rest of the leaf stays
      // the slot to visit (same order, same counts), which keeps lanes at
      // leaves in step with lanes at inner nodes
      const int cnt = left < kTrisPerStep ? left : kTrisPerStep;
      for (int i = 0; i < cnt; ++i) {
        const float4* tp = p.tris + 3 * (long long)(first + i);
        const float4 A = __ldg(tp), E1 = __ldg(tp + 1), E2 = __ldg(tp + 2);
        ++s.ttest;
        float t, u, v;
        if (tri_test(A, E1, E2, s.ox, s.oy, s.oz, s.dx, s.dy, s.dz, s.tmin, s.tcur, t, u, v)) {
          record_accept<OPT>(s, t, u, v, A, first + i);
          if (MODE == 1) {
            done = true;
            break;
          }
          s.tcur = t;
        }
      }
      if (!done && left > cnt) {
        s.cur = kLeaf | ((uint32_t)(left - cnt - 1) << 28) | (uint32_t)(first + cnt);
      } else {
        s.have = false;
      }
    } else if constexpr (kDefer) {
      const float4* nd = p.nodes + (long long)s.cur * p.node_f4;
      Rec rc;
      load_rec<true>(p, s.cur, rc);
      return trace_inner_deferred<RR, STACK>(p, s, stack, tstack, nd, rc);
    } else {
      const float4* nd = p.nodes + (long long)s.cur * p.node_f4;
      Rec rc;
      if constexpr (kSpec) {
        // the prefetch holds the first 64 bytes; the scales follow in the
        // same lines and are requested here, used after the slab tests
        if (!s.pre) load_rec<false>(p, s.cur, s.nx);
        rc = s.nx;
        if constexpr (kScaled) {
          rc.f4 = __ldg(nd + 4);
          rc.f5 = __ldg(nd + 5);
        }
        s.pre = false;
      } else {
        load_rec<kScaled && (OPT & OPT_LAZY) == 0>(p, s.cur, rc);
      }
      const float4 f0 = rc.f0, f1 = rc.f1, f2 = rc.f2;
      const uint4 f3 = make_uint4(__float_as_uint(rc.f3.x), __float_as_uint(rc.f3.y),
                                  __float_as_uint(rc.f3.z), __float_as_uint(rc.f3.w));
      s.ntest += 2;
      const float lo0[3] = {f0.x, f0.y, f2.x}, hi0[3] = {f0.z, f0.w, f2.y};
      const float lo1[3] = {f1.x, f1.y, f2.z}, hi1[3] = {f1.z, f1.w, f2.w};
      const float o[3] = {s.ox, s.oy, s.oz};
      float tn[2], tf[2];
      bool hit[2];
      slab2(f0, f1, f2, s.ox, s.oy, s.oz, s.ix, s.iy, s.iz, s.tmin, s.tcur, tn, tf, hit);
      const uint32_t s0 = f3.x, s1 = f3.y;
      uint32_t spec_slot = kLeaf;  // a leaf word: nothing fetched
      if constexpr (CULL != 0) {
        const float d[3] = {s.dx, s.dy, s.dz};
        const bool need0 = hit[0] && !(f3.z & kMetaFull);
        const bool need1 = hit[1] && !(f3.w & kMetaFull);
        if constexpr (kScaled && !kSpec && (OPT & OPT_LAZY) != 0) {
          if (need0 || need1) {
            rc.f4 = __ldg(nd + 4);
            rc.f5 = __ldg(nd + 5);
          }
        }
        float sc[2][3];
        if constexpr (SCALES) {
          sc[0][0] = rc.f4.x; sc[0][1] = rc.f4.y; sc[0][2] = rc.f5.x;
          sc[1][0] = rc.f4.z; sc[1][1] = rc.f4.w; sc[1][2] = rc.f5.y;
        } else {
#pragma unroll
          for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int k = 0; k < 3; ++k)
              sc[c][k] = scale_of<RR>(c ? lo1[k] : lo0[k], c ? hi1[k] : hi0[k]);
        }
        const uint8_t* objs = reinterpret_cast<const uint8_t*>(nd + p.mask_off_f4);
        if constexpr (kSplit) {
          Lookup<RR, CULL, LUTV> L0, L1;
          if (need0) lookup_issue<RR, CULL, LUTV, OPT>(p, L0, objs, f3.z, lo0, sc[0], o, d, tn[0], tf[0]);
          if (need1)
            lookup_issue<RR, CULL, LUTV, OPT>(p, L1, objs + MB, f3.w, lo1, sc[1], o, d, tn[1], tf[1]);
          if constexpr (kSpec) {
            // the child visited next if both survive their tests
            if (hit[0] || hit[1]) {
              const int c = (hit[0] && hit[1]) ? (tn[1] < tn[0] ? 1 : 0) : (hit[0] ? 0 : 1);
              const uint32_t sl = c ? s1 : s0;
              if (!(sl & kLeaf) && slot_ok(sl, (long long)s.cur, p)) {
                spec_slot = sl;
                load_rec<false>(p, sl, s.nx);
              }
            }
          }
          if (need0) hit[0] = lookup_result(L0);
          if (need1) hit[1] = lookup_result(L1);
        } else {
          if (need0)
            hit[0] = cull_test<RR, CULL, LUTV, OPT>(p, sh, objs, f3.z, lo0, sc[0], o, d, tn[0], tf[0]);
          if (need1)
            hit[1] =
                cull_test<RR, CULL, LUTV, OPT>(p, sh, objs + MB, f3.w, lo1, sc[1], o, d, tn[1], tf[1]);
        }
      }
      if ((hit[0] && !slot_ok(s0, (long long)s.cur, p)) ||
          (hit[1] && !slot_ok(s1, (long long)s.cur, p))) {
        atomicOr(p.status, (unsigned)ST_BAD_NODE);
        done = true;
      } else if (hit[0] && hit[1]) {
        const int nr = tn[1] < tn[0] ? 1 : 0;
        if (stack_push<STACK, OPT>(s, stack,
                                   make_uint2(nr ? s0 : s1, __float_as_uint(nr ? tn[0] : tn[1])))) {
          s.cur = nr ? s1 : s0;
        } else {
          atomicOr(p.status, (unsigned)ST_STACK);
          done = true;
        }
      } else if (hit[0]) {
        s.cur = s0;
      } else if (hit[1]) {
        s.cur = s1;
      } else {
        s.have = false;
      }
      if constexpr (kSpec) s.pre = !(spec_slot & kLeaf) && s.have && s.cur == spec_slot;
    }
  }
  if (!done && !s.have) done = pop_next<OPT>(s, stack, tstack);
  if constexpr (kSpec) {
    // the next inner record is requested now, before the loop's bookkeeping
    if (!done && s.have && !s.pre && !(s.cur & kLeaf) && (long long)s.cur < p.num_nodes) {
      load_rec<false>(p, s.cur, s.nx);
      s.pre = true;
    }
  }
  return done;
}

constexpr uint32_t kNoSlot = 0xFFFFFFFFu;

// One traversal step on 4-wide nodes (SC_LAYOUT_PLAIN4 / MASKED4): a leaf
// as in trace_step, or one node: the slab tests of its (2..4) children,
// their culling tests, then the slab-passing children ordered by entry
// distance (ties by position); the nearest is visited next, the others
// pushed farthest first.  Counts: node_tests += the node's children.
template <int R, int CULL, int MODE, int LUTV, int SCALES, int STACK = kStack, int OPT = 0>
__device__ __forceinline__ bool trace_step4(const Params& p, RayState& s, uint2* stack,
                                            const SharedTables<(R > 0 ? R : 4), LUTV>& sh) {
  static_assert((OPT & (OPT_PAIR | OPT_SPEC | OPT_TOS | OPT_SSTACK)) == 0,
                "binary-step options only");
  constexpr int RR = (R > 0 ? R : 4);
  constexpr int MB = MaskTraits<RR>::kStrideBytes;
  bool done = false;
  if (s.have) {
    if (s.cur & kLeaf) {
      const int first = (int)(s.cur & 0x0FFFFFFFu);
      const int left = (int)((s.cur >> 28) & 7u) + 1;
      const int cnt = left < kTrisPerStep ? left : kTrisPerStep;
      for (int i = 0; i < cnt; ++i) {
        const float4* tp = p.tris + 3 * (long long)(first + i);
        const float4 A = __ldg(tp), E1 = __ldg(tp + 1), E2 = __ldg(tp + 2);
        ++s.ttest;
        float t, u, v;
        if (tri_test(A, E1, E2, s.ox, s.oy, s.oz, s.dx, s.dy, s.dz, s.tmin, s.tcur, t, u, v)) {
          record_accept<OPT>(s, t, u, v, A, first + i);
          if (MODE == 1) {
            done = true;
            break;
          }
          s.tcur = t;
        }
      }
      if (!done && left > cnt) {
        s.cur = kLeaf | ((uint32_t)(left - cnt - 1) << 28) | (uint32_t)(first + cnt);
      } else {
        s.have = false;
      }
    } else {
      const float4* nd = p.nodes + (long long)s.cur * p.node_f4;
      const uint4 sl = __ldg(reinterpret_cast<const uint4*>(nd + 6));
      const uint32_t slot[4] = {sl.x, sl.y, sl.z, sl.w};
      // slab tests one axis at a time over the four children: only one
      // axis's bounds are live at once.  The min / max grouping is the
      // binary step's: tn = max(max(near_x, near_y), max(near_z, tmin)),
      // tf = min(min(far_x, far_y), min(far_z, tcur)).
      float tn[4], tf[4];
      {
        const float4 l = __ldg(nd), h = __ldg(nd + 3);
        const float lv[4] = {l.x, l.y, l.z, l.w}, hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float a0 = __fmul_rn(__fsub_rn(lv[c], s.ox), s.ix);
          const float a1 = __fmul_rn(__fsub_rn(hv[c], s.ox), s.ix);
          tn[c] = fminf(a0, a1);
          tf[c] = fmaxf(a0, a1);
        }
      }
      {
        const float4 l = __ldg(nd + 1), h = __ldg(nd + 4);
        const float lv[4] = {l.x, l.y, l.z, l.w}, hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float a0 = __fmul_rn(__fsub_rn(lv[c], s.oy), s.iy);
          const float a1 = __fmul_rn(__fsub_rn(hv[c], s.oy), s.iy);
          tn[c] = fmaxf(tn[c], fminf(a0, a1));
          tf[c] = fminf(tf[c], fmaxf(a0, a1));
        }
      }
      bool hit[4];
      {
        const float4 l = __ldg(nd + 2), h = __ldg(nd + 5);
        const float lv[4] = {l.x, l.y, l.z, l.w}, hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float a0 = __fmul_rn(__fsub_rn(lv[c], s.oz), s.iz);
          const float a1 = __fmul_rn(__fsub_rn(hv[c], s.oz), s.iz);
          tn[c] = fmaxf(tn[c], fmaxf(fminf(a0, a1), s.tmin));
          tf[c] = fminf(tf[c], fminf(fmaxf(a0, a1), s.tcur));
          hit[c] = slot[c] != kNoSlot && tn[c] <= __fmul_rn(tf[c], kRobust);
        }
      }
      s.ntest += (slot[2] != kNoSlot ? 1u : 0u) + (slot[3] != kNoSlot ? 1u : 0u) + 2u;
      if constexpr (CULL != 0) {
        const uint4 me = __ldg(reinterpret_cast<const uint4*>(nd + 7));
        const unsigned meta[4] = {me.x, me.y, me.z, me.w};
        unsigned need = 0u;
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (hit[c] && !(meta[c] & kMetaFull)) need |= 1u << c;
        if (need) {
          const float o[3] = {s.ox, s.oy, s.oz};
          const float d[3] = {s.dx, s.dy, s.dz};
          const float* rec = reinterpret_cast<const float*>(nd);
          const uint8_t* objs = reinterpret_cast<const uint8_t*>(nd + p.mask_off_f4);
          // one test per needed child; a lane runs only its own.  The
          // child's lower corner and scales are read again from the record
          // (float c of rows 0..2 and 8..10), already in L1.
          while (need) {
            const int c = __ffs(need) - 1;
            need &= need - 1u;
            const float l3[3] = {__ldg(rec + c), __ldg(rec + 4 + c), __ldg(rec + 8 + c)};
            const float s3[3] = {__ldg(rec + 32 + c), __ldg(rec + 36 + c), __ldg(rec + 40 + c)};
            const float tnc = c == 0 ? tn[0] : c == 1 ? tn[1] : c == 2 ? tn[2] : tn[3];
            const float tfc = c == 0 ? tf[0] : c == 1 ? tf[1] : c == 2 ? tf[2] : tf[3];
            const unsigned mc = c == 0 ? meta[0] : c == 1 ? meta[1] : c == 2 ? meta[2] : meta[3];
            if (!cull_test<RR, CULL, LUTV, OPT>(p, sh, objs + c * MB, mc, l3, s3, o, d, tnc, tfc)) {
              if (c == 0) hit[0] = false;
              else if (c == 1) hit[1] = false;
              else if (c == 2) hit[2] = false;
              else hit[3] = false;
            }
          }
        }
      }
      // order the surviving children by (tn, position)
      int ord[4];
      int nh = 0;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (!hit[c]) continue;
        if (!slot_ok(slot[c], (long long)s.cur, p)) {
          atomicOr(p.status, (unsigned)ST_BAD_NODE);
          done = true;
        }
        int j = nh++;
        while (j > 0 && tn[ord[j - 1]] > tn[c]) {
          ord[j] = ord[j - 1];
          --j;
        }
        ord[j] = c;
      }
      if (!done) {
        if (nh == 0) {
          s.have = false;
        } else if (s.sp + nh - 1 > STACK) {
          atomicOr(p.status, (unsigned)ST_STACK);
          done = true;
        } else {
          for (int j = nh - 1; j >= 1; --j) {
            stack[s.sp] = make_uint2(slot[ord[j]], __float_as_uint(tn[ord[j]]));
            ++s.sp;
          }
          s.cur = slot[ord[0]];
        }
      }
    }
  }
  if (!done && !s.have) {
    while (s.sp > 0) {
      --s.sp;
      if (__uint_as_float(stack[s.sp].y) > __fmul_rn(s.tcur, kRobust)) continue;
      s.cur = stack[s.sp].x;
      s.have = true;
      break;
    }
    if (!s.have) done = true;
  }
  return done;
}

// The step of a trace or wave kernel of the given node width.
template <int WIDTH, int R, int CULL, int MODE, int LUTV, int SCALES, int STACK, int OPT = 0>
__device__ __forceinline__ bool step_w(const Params& p, RayState& s, uint2* stack,
                                       const SharedTables<(R > 0 ? R : 4), LUTV>& sh,
                                       uint32_t* tstack) {
  if constexpr (WIDTH == 4) {
    return trace_step4<R, CULL, MODE, LUTV, SCALES, STACK, OPT>(p, s, stack, sh);
  } else {
    return trace_step<R, CULL, MODE, LUTV, SCALES, STACK, OPT>(p, s, stack, sh, tstack);
  }
}

// Warp-level ray fetch: once at least `refill` lanes are idle (or all are),
// the warp takes that many ray indices with one atomicAdd; returns the index
// for this lane (or -1).  `exhausted` turns warp-uniformly true once the
// counter has passed n.
__device__ __forceinline__ long long warp_fetch(bool active, unsigned* counter, long long n,
                                                int refill, bool& exhausted) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned idle = __ballot_sync(0xffffffffu, !active);
  if (idle == 0u || exhausted || (__popc(idle) < refill && idle != 0xffffffffu)) return -1;
  const int leader = __ffs(idle) - 1;
  unsigned base = 0;
  if ((int)lane == leader) base = atomicAdd(counter, (unsigned)__popc(idle));
  base = __shfl_sync(0xffffffffu, base, leader);
  if ((long long)base + __popc(idle) >= n) exhausted = true;
  if (active) return -1;
  const long long r = (long long)base + __popc(idle & ((1u << lane) - 1u));
  return r < n ? r : -1;
}

// CULL: 0 plain, 1 uncompressed masks, 2 compressed masks.  MODE: 0 closest,
// 1 any.  LUTV: 0 full table in global memory (one entry per lookup through
// L1/L2), 1 factored tables in shared memory, 2 (compressed only) the
// precomputed bit table of Sec. 3.2.2 (one bit per ray mask and LUT entry),
// 3 (R = 4 only) the full table and the LUT in shared memory, 4
// (uncompressed, R = 4 or 6) the R_ray = 2R table in global memory.
// SCALES: 1 = the per-child Alg. 1 scales R/extent are precomputed in the
// node record, 0 = divided.
template <int R, int CULL, int MODE, int LUTV, int SCALES, int WIDTH = 2, int OPT = 0>
__global__ void __launch_bounds__(kBlock) trace_kernel(Params p) {
  constexpr int RR = (R > 0 ? R : 4);
  __shared__ SharedTables<RR, LUTV> sh;
  if constexpr (CULL != 0) {
    stage_tables(sh, p);
    __syncthreads();
  }
  uint2 stack[kStack];
  uint32_t tstack[(OPT & OPT_DEFER) ? kStack : 1];
  RayState s;
  s.have = false;
  long long rid = -1;
  bool active = false, exhausted = false;
  for (;;) {
    const long long r = warp_fetch(active, &p.work[0], p.n, p.refill, exhausted);
    if (r >= 0) {
      rid = r;
      active = true;
      ray_init(s, __ldg(&p.rays[2 * r]), __ldg(&p.rays[2 * r + 1]), p);
    }
    if (!__any_sync(0xffffffffu, active)) break;
    if (!active) continue;
    if (step_w<WIDTH, R, CULL, MODE, LUTV, SCALES, kStack, OPT>(p, s, stack, sh, tstack)) {
      p.hits[rid] = hit_record<OPT>(s);
      if (p.counts) p.counts[rid] = make_uint2(s.ntest, s.ttest);
      active = false;
    }
  }
}

// ------------------------------------------------------------------ waves --

constexpr int kMaxWaves = 5;  // primary + up to 4 bounces
constexpr int kWaveMinBlocks = 8;  // register bound of the wave kernel (<= 72 / thread)

// Control words of the wave workspace (uint32 indices): a head, then 16
// words per chunk of primary rays.
enum {
  WW_STATUS = 16,
  WW_BAR_COUNT = 24,
  WW_BAR_GEN = 25,
  WW_NCHUNKS = 32,     // written by the kernel: chunks of this launch
  WW_HEAD = 64,        // chunk c's words start at WW_HEAD + 16 c:
  WW_FETCH = 0,        //   [0, kMaxWaves): ray counters of each wave
  WW_SIZE = 8,         //   [8, 8 + kMaxWaves): rays appended to each wave
  WW_CHUNK_WORDS = 16
};
enum { ST_TIMEOUT = 4 };

// Bounce-queue sort (OPT_SORT): key = direction octant (3 bits) above the
// Morton code of the origin's cell in a 16^3 grid over the scene box.
constexpr int kSortCellBits = 4;
constexpr int kSortBins = 8 << (3 * kSortCellBits);

struct WaveParams {
  Params p;                    // image, status word (p.work = control words), refill
  const float4* rays0;         // primary rays
  long long n0;
  long long chunk;             // primary rays per chunk (the wave size)
  float4* qrays[2];            // bounce-ray queues (scratch), `chunk` rays each
  int* qpath[2];               // path id of each queued ray
  float4* srays;               // OPT_SORT: sorted queue (scratch), `chunk` rays
  int* spath;                  //   its path ids
  unsigned* hist;              //   kSortBins counters / offsets
  float box_lo[3];             //   scene box lower corner
  float box_scale[3];          //   2^kSortCellBits / extent per axis
  float4* hits[kMaxWaves];     // per wave: {t, id, u, v}
  int* path[kMaxWaves];        // per wave: path id (primary ray index)
  uint2* counts[kMaxWaves];    // per wave, optional
  float4* orays[kMaxWaves];    // per wave, optional: the traced rays
  int bounces;
  unsigned seed;
  unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident).  The
// wait is bounded: after timeout_ns the block records ST_TIMEOUT and
// returns false, so a kernel can never hang here.
__device__ __forceinline__ bool grid_barrier(unsigned* w, unsigned long long timeout_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = &w[WW_BAR_GEN];
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&w[WW_BAR_COUNT], 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&w[WW_BAR_COUNT], 0u);
      __threadfence();
      atomicAdd(&w[WW_BAR_GEN], 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == g) {
        if (global_ns() - t0 > timeout_ns) {
          atomicOr(&w[WW_STATUS], (unsigned)ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ unsigned sort_key(const float4 a, const float4 b, const WaveParams& wp) {
  const unsigned oct = (b.x < 0.0f ? 1u : 0u) | (b.y < 0.0f ? 2u : 0u) | (b.z < 0.0f ? 4u : 0u);
  constexpr int kMax = (1 << kSortCellBits) - 1;
  const float o[3] = {a.x, a.y, a.z};
  unsigned c[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int v = __float2int_rz((o[k] - wp.box_lo[k]) * wp.box_scale[k]);
    c[k] = (unsigned)min(max(v, 0), kMax);
  }
  unsigned m = 0;
#pragma unroll
  for (int bit = 0; bit < kSortCellBits; ++bit)
    m |= (((c[0] >> bit) & 1u) << (3 * bit)) | (((c[1] >> bit) & 1u) << (3 * bit + 1)) |
         (((c[2] >> bit) & 1u) << (3 * bit + 2));
  return (oct << (3 * kSortCellBits)) | m;
}

// Counting sort of queue (q, qp) of n rays into (wp.srays, wp.spath) by
// sort_key, across the whole cooperative grid; wp.hist must be zero on
// entry.  Three bounded grid barriers; false if one timed out.
template <int BLOCK>
__device__ bool sort_queue(const WaveParams& wp, const float4* q, const int* qp, long long n) {
  const long long tid = (long long)blockIdx.x * BLOCK + threadIdx.x;
  const long long nth = (long long)gridDim.x * BLOCK;
  for (long long i = tid; i < n; i += nth)
    atomicAdd(&wp.hist[sort_key(__ldcg(&q[2 * i]), __ldcg(&q[2 * i + 1]), wp)], 1u);
  __threadfence();
  if (!grid_barrier(wp.p.work, wp.timeout_ns)) return false;
  if (blockIdx.x == 0) {
    // exclusive scan in place: each thread a contiguous run of bins
    constexpr int kPer = kSortBins / BLOCK;
    __shared__ unsigned part[BLOCK];
    unsigned sum = 0;
    for (int j = 0; j < kPer; ++j) sum += __ldcg(&wp.hist[threadIdx.x * kPer + j]);
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned acc = 0;
      for (int t = 0; t < BLOCK; ++t) {
        const unsigned v = part[t];
        part[t] = acc;
        acc += v;
      }
    }
    __syncthreads();
    unsigned acc = part[threadIdx.x];
    for (int j = 0; j < kPer; ++j) {
      unsigned* h = &wp.hist[threadIdx.x * kPer + j];
      const unsigned v = __ldcg(h);
      __stcg(h, acc);
      acc += v;
    }
  }
  __threadfence();
  if (!grid_barrier(wp.p.work, wp.timeout_ns)) return false;
  for (long long i = tid; i < n; i += nth) {
    const float4 a = __ldcg(&q[2 * i]), b = __ldcg(&q[2 * i + 1]);
    const unsigned pos = atomicAdd(&wp.hist[sort_key(a, b, wp)], 1u);
    if ((long long)pos < n) {  // always: the offsets of a full count
      wp.srays[2 * (long long)pos] = a;
      wp.srays[2 * (long long)pos + 1] = b;
      wp.spath[pos] = __ldcg(&qp[i]);
    }
  }
  __threadfence();
  return grid_barrier(wp.p.work, wp.timeout_ns);
}

// Diffuse bounce ray from a hit (same canonical op sequence as the CPU
// reference): origin o + t d; geometric normal cross(e1, e2) turned against
// d and normalised; frame by cross products; unit-disk point by rejection
// (<= 64 tries, else the centre) lifted to the hemisphere.  Random bits:
// hash of (seed, path id, bounce, k) after Jarzynski & Olano (JCGT 2020).
__device__ __forceinline__ unsigned pcg_hash(unsigned v) {
  const unsigned state = v * 747796405u + 2891336453u;
  const unsigned word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
  return (word >> 22u) ^ word;
}

// Scalars by value (not the ray state by reference): the call is out of
// line, and taking the state's address would pin it in local memory.
static __device__ __noinline__ bool make_bounce(float ox, float oy, float oz, float dx, float dy,
                                                float dz, float ht, const float4 E1,
                                                const float4 E2, unsigned seed, unsigned path,
                                                unsigned bounce, float4& r0, float4& r1) {
  const float px = __fadd_rn(ox, __fmul_rn(ht, dx));
  const float py = __fadd_rn(oy, __fmul_rn(ht, dy));
  const float pz = __fadd_rn(oz, __fmul_rn(ht, dz));
  float nx = __fsub_rn(__fmul_rn(E1.y, E2.z), __fmul_rn(E1.z, E2.y));
  float ny = __fsub_rn(__fmul_rn(E1.z, E2.x), __fmul_rn(E1.x, E2.z));
  float nz = __fsub_rn(__fmul_rn(E1.x, E2.y), __fmul_rn(E1.y, E2.x));
  if (__fadd_rn(__fadd_rn(__fmul_rn(nx, dx), __fmul_rn(ny, dy)), __fmul_rn(nz, dz)) > 0.0f) {
    nx = -nx; ny = -ny; nz = -nz;
  }
  const float l2 = __fadd_rn(__fadd_rn(__fmul_rn(nx, nx), __fmul_rn(ny, ny)), __fmul_rn(nz, nz));
  if (!(l2 > 0.0f)) return false;
  const float l = __fsqrt_rn(l2);
  nx = __fdiv_rn(nx, l); ny = __fdiv_rn(ny, l); nz = __fdiv_rn(nz, l);
  const float ax = fabsf(nx) > 0.9f ? 0.0f : 1.0f, ay = fabsf(nx) > 0.9f ? 1.0f : 0.0f, az = 0.0f;
  float t1x = __fsub_rn(__fmul_rn(ay, nz), __fmul_rn(az, ny));
  float t1y = __fsub_rn(__fmul_rn(az, nx), __fmul_rn(ax, nz));
  float t1z = __fsub_rn(__fmul_rn(ax, ny), __fmul_rn(ay, nx));
  const float m = __fsqrt_rn(
      __fadd_rn(__fadd_rn(__fmul_rn(t1x, t1x), __fmul_rn(t1y, t1y)), __fmul_rn(t1z, t1z)));
  t1x = __fdiv_rn(t1x, m); t1y = __fdiv_rn(t1y, m); t1z = __fdiv_rn(t1z, m);
  const float t2x = __fsub_rn(__fmul_rn(ny, t1z), __fmul_rn(nz, t1y));
  const float t2y = __fsub_rn(__fmul_rn(nz, t1x), __fmul_rn(nx, t1z));
  const float t2z = __fsub_rn(__fmul_rn(nx, t1y), __fmul_rn(ny, t1x));
  const unsigned key = pcg_hash(pcg_hash(seed ^ (bounce << 24)) + path);
  float x = 0.0f, y = 0.0f, r2 = 0.0f;
  for (unsigned k = 0; k < 64; ++k) {
    const float u1 = __fmul_rn((float)(pcg_hash(key + 2 * k) >> 8), 5.9604644775390625e-08f);
    const float u2 = __fmul_rn((float)(pcg_hash(key + 2 * k + 1) >> 8), 5.9604644775390625e-08f);
    const float xx = __fsub_rn(__fmul_rn(2.0f, u1), 1.0f);
    const float yy = __fsub_rn(__fmul_rn(2.0f, u2), 1.0f);
    const float rr = __fadd_rn(__fmul_rn(xx, xx), __fmul_rn(yy, yy));
    if (rr < 1.0f) {
      x = xx; y = yy; r2 = rr;
      break;
    }
  }
  const float z = __fsqrt_rn(__fsub_rn(1.0f, r2));
  r0 = make_float4(px, py, pz, 1e-4f);
  r1 = make_float4(__fadd_rn(__fadd_rn(__fmul_rn(x, t1x), __fmul_rn(y, t2x)), __fmul_rn(z, nx)),
                   __fadd_rn(__fadd_rn(__fmul_rn(x, t1y), __fmul_rn(y, t2y)), __fmul_rn(z, ny)),
                   __fadd_rn(__fadd_rn(__fmul_rn(x, t1z), __fmul_rn(y, t2z)), __fmul_rn(z, nz)),
                   __int_as_float(0x7f800000));
  return true;
}

// All waves in one cooperative persistent launch.  The primary rays are
// taken in chunks of `chunk` rays (the wave size); for each chunk, wave 0
// traces its primary rays and every hit of wave w < bounces appends its
// bounce ray to the queue of wave w + 1 (warp-aggregated atomicAdd, so a
// queue holds only spawned rays: compacted).  A bounded grid barrier
// separates the waves.  Outputs: wave 0 by primary index; wave w >= 1 after
// the entries of the previous chunks.  The blocks resident per SM (the
// register bound) are kWaveMinBlocks of kBlock threads unless OPT_OCC9 /
// OPT_OCC10 raise them.
template <int OPT>
constexpr int kWaveBlocksPerSM =
    kWaveMinBlocks + ((OPT & OPT_OCC10) ? 2 : ((OPT & OPT_OCC9) ? 1 : 0));

template <int R, int CULL, int LUTV, int SCALES, int BLOCK = kBlock, int STACK = kStack,
          int WIDTH = 2, int OPT = 0>
__global__ void __launch_bounds__(BLOCK, kWaveBlocksPerSM<OPT> * kBlock / BLOCK)
    waves_kernel(WaveParams wp) {
  static_assert(BLOCK <= kMaxBlock, "the hit slots hold kMaxBlock threads");
  constexpr int RR = (R > 0 ? R : 4);
  __shared__ SharedTables<RR, LUTV> sh;
  const Params& p = wp.p;
  if constexpr (CULL != 0) {
    stage_tables(sh, p);
    __syncthreads();
  }
  const unsigned lane = threadIdx.x & 31u;
  if (blockIdx.x == 0 && threadIdx.x == 0)
    p.work[WW_NCHUNKS] = (unsigned)((wp.n0 + wp.chunk - 1) / wp.chunk);
  uint2 stack[STACK];
  uint32_t tstack[(OPT & OPT_DEFER) ? STACK : 1];
  long long ci = 0;
  for (long long c0 = 0; c0 < wp.n0; c0 += wp.chunk, ++ci) {
    unsigned* cw = p.work + WW_HEAD + WW_CHUNK_WORDS * ci;
    const long long nc = (wp.n0 - c0 < wp.chunk) ? wp.n0 - c0 : wp.chunk;
    for (int w = 0; w <= wp.bounces; ++w) {
      const long long n = (w == 0) ? nc : (long long)(*(volatile unsigned*)&cw[WW_SIZE + w]);
      long long out_base = c0;
      if (w > 0) {
        out_base = 0;
        for (long long c = 0; c < ci; ++c)
          out_base += *(volatile unsigned*)&p.work[WW_HEAD + WW_CHUNK_WORDS * c + WW_SIZE + w];
      }
      const float4* rays = (w == 0) ? wp.rays0 + 2 * c0 : wp.qrays[w & 1];
      const int* qpath = (w == 0) ? nullptr : wp.qpath[w & 1];
      if constexpr ((OPT & OPT_SORT) != 0) {
        if (w > 0) {
          if (!sort_queue<BLOCK>(wp, rays, qpath, n)) return;
          rays = wp.srays;
          qpath = wp.spath;
        }
        if (w < wp.bounces) {
          // zero the counters for the sort before the next wave (the barrier
          // at the end of this wave orders it before the count)
          for (long long i = (long long)blockIdx.x * BLOCK + threadIdx.x; i < kSortBins;
               i += (long long)gridDim.x * BLOCK)
            wp.hist[i] = 0u;
        }
      }
      RayState s;
      s.have = false;
      long long rid = -1;
      bool active = false, exhausted = false;
      for (;;) {
        const long long r = warp_fetch(active, &cw[WW_FETCH + w], n, p.refill, exhausted);
        if (r >= 0) {
          rid = r;
          active = true;
          // queued rays were written by other SMs in this launch: read them
          // through L2 (ld.global.cg), never through the read-only / L1 path
          ray_init(s, __ldcg(&rays[2 * r]), __ldcg(&rays[2 * r + 1]), p);
        }
        if (!__any_sync(0xffffffffu, active)) break;
        const bool done =
            active && step_w<WIDTH, R, CULL, 0, LUTV, SCALES, STACK, OPT>(p, s, stack, sh, tstack);
        if (!__any_sync(0xffffffffu, done)) continue;
        bool spawn = false;
        float4 b0, b1;
        unsigned pid = 0;
        if (done) {
          pid = qpath ? (unsigned)__ldcg(&qpath[rid]) : (unsigned)(c0 + rid);
          const long long o = out_base + rid;
          wp.hits[w][o] = hit_record<OPT>(s);
          if (wp.path[w]) wp.path[w][o] = (int)pid;
          if (wp.counts[w]) wp.counts[w][o] = make_uint2(s.ntest, s.ttest);
          if (wp.orays[w]) {
            wp.orays[w][2 * o] = __ldcg(&rays[2 * rid]);
            wp.orays[w][2 * o + 1] = __ldcg(&rays[2 * rid + 1]);
          }
          if (w < wp.bounces && s.hpos >= 0) {
            const float4* tp = p.tris + 3 * (long long)s.hpos;
            spawn = make_bounce(s.ox, s.oy, s.oz, s.dx, s.dy, s.dz, s.ht, __ldg(tp + 1),
                                __ldg(tp + 2), wp.seed, pid, (unsigned)(w + 1), b0, b1);
          }
          active = false;
        }
        const unsigned sm = __ballot_sync(0xffffffffu, spawn);
        if (sm) {
          const int leader = __ffs(sm) - 1;
          unsigned base = 0;
          if ((int)lane == leader) base = atomicAdd(&cw[WW_SIZE + w + 1], (unsigned)__popc(sm));
          base = __shfl_sync(0xffffffffu, base, leader);
          if (spawn) {
            const unsigned pos = base + __popc(sm & ((1u << lane) - 1u));
            float4* q = wp.qrays[(w + 1) & 1];
            q[2 * pos] = b0;
            q[2 * pos + 1] = b1;
            wp.qpath[(w + 1) & 1][pos] = (int)pid;
          }
        }
      }
      const bool last = (w == wp.bounces) && (c0 + wp.chunk >= wp.n0);
      if (!last) {
        __threadfence();
        if (!grid_barrier(p.work, wp.timeout_ns)) return;
      }
    }
  }
}

// Slab test of one box (lo = b0.xyz, hi = (b0.w, b1.x, b1.y)) on [tmin,
// tmax], in the same arithmetic as the child tests of trace_step.
__device__ __forceinline__ bool box_hit(const RayState& s, const float4 b0, const float4 b1,
                                        float tmax) {
  const float lo[3] = {b0.x, b0.y, b0.z}, hi[3] = {b0.w, b1.x, b1.y};
  const float o[3] = {s.ox, s.oy, s.oz}, inv[3] = {s.ix, s.iy, s.iz};
  float a0[3], a1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    a0[k] = __fmul_rn(__fsub_rn(lo[k], o[k]), inv[k]);
    a1[k] = __fmul_rn(__fsub_rn(hi[k], o[k]), inv[k]);
  }
  const float tn = fmaxf(fmaxf(fminf(a0[0], a1[0]), fminf(a0[1], a1[1])),
                         fmaxf(fminf(a0[2], a1[2]), s.tmin));
  const float tf = fminf(fminf(fmaxf(a0[0], a1[0]), fmaxf(a0[1], a1[1])),
                         fminf(fmaxf(a0[2], a1[2]), tmax));
  return tn <= __fmul_rn(tf, kRobust);
}

// Seeded closest-hit traversal (learned proposal; not in the paper).
// frontier: entries of 2 float4 = box lo.xyz, hi.x | hi.yz, slot word, 0.
// A class outside [0, nfront) traces the ray without a seed.  Otherwise
// the seed box is slab-tested with the ray's t_max (one node test); if the
// ray enters it, phase 1 traverses the seed subtree with that t_max.
// Phase 2 traverses from the root and skips the seed slot (phase 1 covered
// it, or the ray misses its box).  A phase-1 hit at t_s is held
// provisionally with t_max = nextafter(t_s, +inf), so that an equally
// distant triangle met earlier in traversal order replaces it, and t_max
// drops to t_s when phase 2 reaches the seed slot: the result is the
// plain traversal's closest hit.  Counts sum both phases.
template <int R, int CULL, int LUTV, int SCALES, int OPT = 0>
__global__ void __launch_bounds__(kBlock) seeded_kernel(Params p, const int* cls,
                                                        const float4* frontier, int nfront) {
  constexpr int RR = (R > 0 ? R : 4);
  __shared__ SharedTables<RR, LUTV> sh;
  if constexpr (CULL != 0) {
    stage_tables(sh, p);
    __syncthreads();
  }
  uint2 stack[kStack];
  RayState s;
  s.have = false;
  long long rid = -1;
  float tmax0 = 0.0f;
  int phase = 0, seed_pos = -1;
  uint32_t seed = 0u;
  bool has_seed = false, active = false, exhausted = false;
  for (;;) {
    const long long r = warp_fetch(active, &p.work[0], p.n, p.refill, exhausted);
    if (r >= 0) {
      rid = r;
      active = true;
      const float4 rb = __ldg(&p.rays[2 * r + 1]);
      ray_init(s, __ldg(&p.rays[2 * r]), rb, p);
      tmax0 = rb.w;
      seed_pos = -1;
      has_seed = false;
      phase = 2;
      s.cur = p.root_slot;
      s.have = p.has_root != 0;
      const int c = cls[r];
      if (p.has_root && c >= 0 && c < nfront) {
        const float4 e0 = __ldg(&frontier[2 * c]), e1 = __ldg(&frontier[2 * c + 1]);
        seed = __float_as_uint(e1.z);
        if (!slot_ok(seed, -1, p)) {
          atomicOr(p.status, (unsigned)ST_BAD_NODE);
        } else {
          has_seed = true;
          ++s.ntest;
          if (box_hit(s, e0, e1, tmax0)) {
            phase = 1;
            s.cur = seed;
          }
        }
      }
    }
    if (!__any_sync(0xffffffffu, active)) break;
    if (!active) continue;
    if (phase == 2 && has_seed && s.have && s.cur == seed) {
      if (s.hpos >= 0 && s.hpos == seed_pos) s.tcur = s.ht;  // the seed counts as found here
      s.have = false;
    }
    if (trace_step<R, CULL, 0, LUTV, SCALES, kStack, OPT>(p, s, stack, sh)) {
      if (phase == 1) {
        phase = 2;
        s.sp = 0;
        s.cur = p.root_slot;
        s.have = p.has_root != 0;
        if (s.hpos >= 0) {
          seed_pos = s.hpos;
          s.tcur = nextafterf(s.ht, __int_as_float(0x7f800000));
        } else {
          s.tcur = tmax0;
        }
        continue;
      }
      p.hits[rid] = hit_record<OPT>(s);
      if (p.counts) p.counts[rid] = make_uint2(s.ntest, s.ttest);
      active = false;
    }
  }
}

typedef void (*KernelFn)(Params);
typedef void (*SeededKernelFn)(Params, const int*, const float4*, int);
typedef void (*WaveKernelFn)(WaveParams);

// Block size x stack depth variants of one wave kernel (for the autotuner):
// index [block 64/128/256][stack 32/64].
template <int R, int CULL, int LUTV, int SCALES>
struct WaveVariants {
  static WaveKernelFn get(int block, int stack) {
    static const WaveKernelFn t[3][2] = {
        {waves_kernel<R, CULL, LUTV, SCALES, 64, 32>, waves_kernel<R, CULL, LUTV, SCALES, 64, 64>},
        {waves_kernel<R, CULL, LUTV, SCALES, 128, 32>,
         waves_kernel<R, CULL, LUTV, SCALES, 128, 64>},
        {waves_kernel<R, CULL, LUTV, SCALES, 256, 32>,
         waves_kernel<R, CULL, LUTV, SCALES, 256, 64>}};
    const int bi = block == 64 ? 0 : (block == 256 ? 2 : 1);
    return t[bi][stack == 32 ? 0 : 1];
  }
};

}  // namespace sct
