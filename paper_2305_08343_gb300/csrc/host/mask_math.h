// mask_math.h — the arithmetic of the object masks (Sec. 3.1.1, 3.2.1,
// Alg. 2), shared by the host builder (masks.cpp) and the GPU builder
// (cuda/masks_gpu.cu): one source, compiled for both, so both set the same
// bits.  Double precision, each operation written out in the order of its
// definition (built without FMA contraction on either side).  The GPU
// builder first tries each SAT test with an FP32 filter that decides only
// where the FP64 result is certain (below); on the host, where FP64 is as
// fast as FP32, the FP64 test runs directly.
#ifndef SUBCULL_MASK_MATH_H
#define SUBCULL_MASK_MATH_H

#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define SC_HD __host__ __device__ __forceinline__
#else
#define SC_HD inline
#endif

namespace sc {
namespace mm {

SC_HD double mn(double a, double b) { return a < b ? a : b; }
SC_HD double mx(double a, double b) { return a > b ? a : b; }

// Separating-axis triangle/box overlap (Akenine-Moeller 2001); touching
// counts as overlap.  v: 9 doubles.
SC_HD bool tri_box_overlap(const double* v, const double* bmin, const double* bmax) {
  double c[3], h[3], a[3][3];
  for (int k = 0; k < 3; ++k) {
    c[k] = 0.5 * (bmin[k] + bmax[k]);
    h[k] = 0.5 * (bmax[k] - bmin[k]);
  }
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) a[i][k] = v[3 * i + k] - c[k];
  for (int k = 0; k < 3; ++k) {
    if (mn(mn(a[0][k], a[1][k]), a[2][k]) > h[k]) return false;
    if (mx(mx(a[0][k], a[1][k]), a[2][k]) < -h[k]) return false;
  }
  double e[3][3];
  for (int k = 0; k < 3; ++k) {
    e[0][k] = a[1][k] - a[0][k];
    e[1][k] = a[2][k] - a[1][k];
    e[2][k] = a[0][k] - a[2][k];
  }
  const double nx = e[0][1] * e[1][2] - e[0][2] * e[1][1];
  const double ny = e[0][2] * e[1][0] - e[0][0] * e[1][2];
  const double nz = e[0][0] * e[1][1] - e[0][1] * e[1][0];
  const double d = (nx * a[0][0] + ny * a[0][1]) + nz * a[0][2];
  const double rn = (h[0] * fabs(nx) + h[1] * fabs(ny)) + h[2] * fabs(nz);
  if (fabs(d) > rn) return false;
  for (int i = 0; i < 3; ++i) {
    const double ex = e[i][0], ey = e[i][1], ez = e[i][2];
    const double axes[3][3] = {{0.0, ez, -ey}, {-ez, 0.0, ex}, {ey, -ex, 0.0}};
    for (int k = 0; k < 3; ++k) {
      const double* ax = axes[k];
      const double p0 = (ax[0] * a[0][0] + ax[1] * a[0][1]) + ax[2] * a[0][2];
      const double p1 = (ax[0] * a[1][0] + ax[1] * a[1][1]) + ax[2] * a[1][2];
      const double p2 = (ax[0] * a[2][0] + ax[1] * a[2][1]) + ax[2] * a[2][2];
      const double r = (h[0] * fabs(ax[0]) + h[1] * fabs(ax[1])) + h[2] * fabs(ax[2]);
      if (mn(mn(p0, p1), p2) > r || mx(mx(p0, p1), p2) < -r) return false;
    }
  }
  return true;
}

// ---- single-precision filter for tri_box_overlap ----------------------
// FP64 runs at a small fraction of FP32's rate on the GPU, and the SAT
// test above dominates the GPU mask build.  The filter evaluates the same axes
// in FP32, each value carrying a bound on its distance from the exact real
// value of the same expression on the same (double) inputs.  A comparison
// is decided only when its two sides differ by more than their bounds
// (times a safety factor that also covers the rounding of the bounds
// themselves and the far smaller error of the FP64 evaluation); the exact
// comparison, and so the FP64 one, then has the same outcome.  The overlap
// result is "no axis separates", independent of the order of the axes:
// it is decided as "separated" as soon as one axis separates with margin,
// as "overlap" when every axis fails to separate with margin, and left to
// the FP64 test otherwise.

// An FP32 value and a bound on |value - exact|.
struct Ef {
  float v, e;
};
constexpr float kEfU = 5.9604644775390625e-08f;  // 2^-24, unit roundoff
SC_HD Ef ef_exact(float x) { return Ef{x, 0.0f}; }
SC_HD Ef ef_add(Ef a, Ef b) {
  const float v = a.v + b.v;
  return Ef{v, a.e + b.e + kEfU * fabsf(v)};
}
SC_HD Ef ef_sub(Ef a, Ef b) {
  const float v = a.v - b.v;
  return Ef{v, a.e + b.e + kEfU * fabsf(v)};
}
SC_HD Ef ef_mul(Ef a, Ef b) {
  const float v = a.v * b.v;
  return Ef{v, fabsf(a.v) * b.e + fabsf(b.v) * a.e + a.e * b.e + kEfU * fabsf(v)};
}
SC_HD Ef ef_neg(Ef a) { return Ef{-a.v, a.e}; }
SC_HD Ef ef_abs(Ef a) { return Ef{fabsf(a.v), a.e}; }
SC_HD Ef ef_min(Ef a, Ef b) { return Ef{a.v < b.v ? a.v : b.v, a.e > b.e ? a.e : b.e}; }
SC_HD Ef ef_max(Ef a, Ef b) { return Ef{a.v > b.v ? a.v : b.v, a.e > b.e ? a.e : b.e}; }

// x > y: +1 certainly, -1 certainly not, 0 too close to tell (and for
// values so small that their bounds could have underflowed).
SC_HD int ef_gt(Ef x, Ef y) {
  if (fabsf(x.v) < 1e-18f && fabsf(y.v) < 1e-18f) return 0;
  const float margin = (x.e + y.e) * 1.001f + 1e-30f;
  const float d = x.v - y.v;
  return d > margin ? 1 : (-d > margin ? -1 : 0);
}

// One axis: separated when min(p) > r or max(p) < -r.  +1 separated, -1 not
// separated, 0 undecided.
SC_HD int ef_sep(Ef p0, Ef p1, Ef p2, Ef r) {
  const int lo = ef_gt(ef_min(ef_min(p0, p1), p2), r);
  const int hi = ef_gt(ef_neg(r), ef_max(ef_max(p0, p1), p2));
  if (lo > 0 || hi > 0) return 1;
  return (lo < 0 && hi < 0) ? -1 : 0;
}

// The FP32 inputs of one axis: a vertex coordinate relative to the box
// centre, vk - (bmin + bmax) / 2, and the half extent (bmax - bmin) / 2.
// Both are formed in FP64, where the cancellation of nearby coordinates is
// exact enough, then rounded to FP32; the bounds cover both roundings (the
// FP64 ones are at most 2^-52 (|bmin| + |bmax|)).
SC_HD Ef ef_rel(double vk, double bmin, double bmax) {
  const double c = 0.5 * (bmin + bmax);
  const float absk = 4.5e-16f * ((float)fabs(bmin) + (float)fabs(bmax));
  const float af = (float)(vk - c);
  return Ef{af, 2.0f * kEfU * fabsf(af) + absk + 1e-38f};
}
SC_HD Ef ef_half_extent(double bmin, double bmax) {
  const float absk = 4.5e-16f * ((float)fabs(bmin) + (float)fabs(bmax));
  const float hf = (float)(0.5 * (bmax - bmin));
  return Ef{hf, 2.0f * kEfU * fabsf(hf) + absk + 1e-38f};
}

// The 13 axes of tri_box_overlap in FP32 on a[vertex][axis] (vertices
// relative to the box centre) and the half extents h: 1 overlap, 0 none,
// -1 undecided.
SC_HD int tri_box_overlap_ef(const Ef (*a)[3], const Ef* h) {
  bool open = false;  // an axis left undecided
  for (int k = 0; k < 3; ++k) {
    const int s = ef_sep(a[0][k], a[1][k], a[2][k], h[k]);
    if (s > 0) return 0;
    open |= s == 0;
  }
  Ef e[3][3];
  for (int k = 0; k < 3; ++k) {
    e[0][k] = ef_sub(a[1][k], a[0][k]);
    e[1][k] = ef_sub(a[2][k], a[1][k]);
    e[2][k] = ef_sub(a[0][k], a[2][k]);
  }
  const Ef nx = ef_sub(ef_mul(e[0][1], e[1][2]), ef_mul(e[0][2], e[1][1]));
  const Ef ny = ef_sub(ef_mul(e[0][2], e[1][0]), ef_mul(e[0][0], e[1][2]));
  const Ef nz = ef_sub(ef_mul(e[0][0], e[1][1]), ef_mul(e[0][1], e[1][0]));
  const Ef d = ef_add(ef_add(ef_mul(nx, a[0][0]), ef_mul(ny, a[0][1])), ef_mul(nz, a[0][2]));
  const Ef rn = ef_add(ef_add(ef_mul(h[0], ef_abs(nx)), ef_mul(h[1], ef_abs(ny))),
                       ef_mul(h[2], ef_abs(nz)));
  {
    const int s = ef_gt(ef_abs(d), rn);
    if (s > 0) return 0;
    open |= s == 0;
  }
  const Ef zero = ef_exact(0.0f);
  for (int i = 0; i < 3; ++i) {
    const Ef ex = e[i][0], ey = e[i][1], ez = e[i][2];
    const Ef axes[3][3] = {{zero, ez, ef_neg(ey)}, {ef_neg(ez), zero, ex}, {ey, ef_neg(ex), zero}};
    for (int k = 0; k < 3; ++k) {
      const Ef* ax = axes[k];
      Ef p[3];
      for (int j = 0; j < 3; ++j)
        p[j] = ef_add(ef_add(ef_mul(ax[0], a[j][0]), ef_mul(ax[1], a[j][1])),
                      ef_mul(ax[2], a[j][2]));
      const Ef r = ef_add(ef_add(ef_mul(h[0], ef_abs(ax[0])), ef_mul(h[1], ef_abs(ax[1]))),
                          ef_mul(h[2], ef_abs(ax[2])));
      const int s = ef_sep(p[0], p[1], p[2], r);
      if (s > 0) return 0;
      open |= s == 0;
    }
  }
  return open ? -1 : 1;
}

// tri_box_overlap(v, bmin, bmax) through the FP32 filter: 1 overlap, 0 none,
// -1 undecided.
SC_HD int tri_box_overlap_f32(const double* v, const double* bmin, const double* bmax) {
  Ef h[3], a[3][3];
  for (int k = 0; k < 3; ++k) {
    h[k] = ef_half_extent(bmin[k], bmax[k]);
    for (int i = 0; i < 3; ++i) a[i][k] = ef_rel(v[3 * i + k], bmin[k], bmax[k]);
  }
  return tri_box_overlap_ef(a, h);
}

// Grid of one slot: per axis the dilated voxel bounds.
struct Grid {
  int R;
  double eps;
  double lo[3], ext[3];
  double b0[3][8], b1[3][8];
  SC_HD void init(const float* box, int R_, double eps_) {
    R = R_;
    eps = eps_;
    for (int k = 0; k < 3; ++k) {
      init_axis(box, k);
      for (int i = 0; i < R; ++i) init_cell(k, i);
    }
  }
  // the two steps of init, also run entry by entry by the lanes of a warp
  // (R and eps set first, then the axes, then the cells)
  SC_HD void init_axis(const float* box, int k) {
    lo[k] = (double)box[k];
    ext[k] = (double)box[3 + k] - (double)box[k];
  }
  SC_HD void init_cell(int k, int i) {
    b0[k][i] = (lo[k] + (ext[k] * (double)i) / (double)R) - eps;
    b1[k][i] = (lo[k] + (ext[k] * (double)(i + 1)) / (double)R) + eps;
  }
  // Voxels [i0, i1] on axis k whose dilated box may overlap [tlo, thi]; one
  // voxel of margin beyond the eps-widened range keeps this a superset of
  // what the exact test keeps.
  SC_HD void candidates(int k, double tlo, double thi, int& i0, int& i1) const {
    const double w = ext[k] / (double)R;
    if (!(w > 1e-12 * mx(1.0, fabs(lo[k])))) {
      i0 = 0;
      i1 = R - 1;
      return;
    }
    double q0 = floor(((tlo - eps) - lo[k]) / w) - 1.0;
    double q1 = floor(((thi + eps) - lo[k]) / w) + 1.0;
    q0 = mx(0.0, mn(q0, (double)(R - 1)));
    q1 = mx(0.0, mn(q1, (double)(R - 1)));
    i0 = (int)q0;
    i1 = (int)q1;
  }
};

SC_HD void set_bit(uint32_t* m, int bit) { m[bit >> 5] |= 1u << (bit & 31); }
SC_HD bool get_bit(const uint32_t* m, int bit) { return (m[bit >> 5] >> (bit & 31)) & 1u; }

SC_HD void voxelize_tri(const float* t9, const Grid& g, uint32_t* out) {
  double v[9];
  for (int i = 0; i < 9; ++i) v[i] = (double)t9[i];
  int r0[3], r1[3];
  for (int k = 0; k < 3; ++k) {
    const double tlo = mn(mn(v[k], v[3 + k]), v[6 + k]);
    const double thi = mx(mx(v[k], v[3 + k]), v[6 + k]);
    g.candidates(k, tlo, thi, r0[k], r1[k]);
  }
  const int R = g.R;
  for (int z = r0[2]; z <= r1[2]; ++z)
    for (int y = r0[1]; y <= r1[1]; ++y)
      for (int x = r0[0]; x <= r1[0]; ++x) {
        const int bit = x + R * y + R * R * z;
        if (get_bit(out, bit)) continue;
        const double bmin[3] = {g.b0[0][x], g.b0[1][y], g.b0[2][z]};
        const double bmax[3] = {g.b1[0][x], g.b1[1][y], g.b1[2][z]};
        if (tri_box_overlap(v, bmin, bmax)) set_bit(out, bit);
      }
}

// Alg. 2 parent index: min(floor(R * (pos - pLower) / pExtent), R-1), >= 0.
SC_HD int parent_idx(double pos, double plo, double pext, int R) {
  double q = floor(((double)R * (pos - plo)) / pext);
  q = q < 0.0 ? 0.0 : q;
  q = q > (double)(R - 1) ? (double)(R - 1) : q;
  return (int)q;
}

// Alg. 2: the parent cells [lo, hi] on axis k that child border i (of
// 0..R) falls in, the border dilated by eps.
SC_HD void fill_range(const float* pbox, const float* cbox, int k, int i, int R, double eps,
                      int& lo, int& hi) {
  const double cl = (double)cbox[k], cext = (double)cbox[3 + k] - (double)cbox[k];
  const double pl = (double)pbox[k], pext = (double)pbox[3 + k] - (double)pbox[k];
  const double border = cl + (cext * (double)i) / (double)R;
  if (pext > 0.0) {
    lo = parent_idx(border - eps, pl, pext, R);
    hi = parent_idx(border + eps, pl, pext, R);
  } else {
    lo = 0;
    hi = R - 1;
  }
}

// Alg. 2 (fillByApproximatedOccupancy) with borders dilated by eps.
SC_HD void fill_from_child(uint32_t* out, const float* pbox, const uint32_t* cmask,
                           const float* cbox, int R, double eps) {
  int lo_i[3][9], hi_i[3][9];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i <= R; ++i) fill_range(pbox, cbox, k, i, R, eps, lo_i[k][i], hi_i[k][i]);
  for (int z = 0; z < R; ++z)
    for (int y = 0; y < R; ++y)
      for (int x = 0; x < R; ++x) {
        if (!get_bit(cmask, x + R * y + R * R * z)) continue;
        for (int pz = lo_i[2][z]; pz <= hi_i[2][z + 1]; ++pz)
          for (int py = lo_i[1][y]; py <= hi_i[1][y + 1]; ++py)
            for (int px = lo_i[0][x]; px <= hi_i[0][x + 1]; ++px)
              set_bit(out, px + R * py + R * R * pz);
      }
}

// The BVH arrays a slot's mask reads (host vectors or device copies).
struct MaskInputs {
  const float* tris;    // [ntri][9], input order
  const int32_t* perm;  // leaf position -> triangle id
  const int32_t* child; // [nn][2]
  const int32_t* count; // [nn][2]
  const float* box;     // [nn][2][6]
  uint32_t* masks;      // [nn][2][W]
  int R, L, W;
  double eps;
};

SC_HD void leaf_into(const MaskInputs& b, int32_t first, int32_t count, const Grid& g,
                     uint32_t* out) {
  for (int32_t i = 0; i < count; ++i) voxelize_tri(&b.tris[9 * (size_t)b.perm[first + i]], g, out);
}

// Deepest L the builders take (a stack frame per level below a slot).
constexpr int kMaxL = 63;

// Descendants of node m (depth = levels below the slot): leaves fewer than L
// levels below are voxelized, descendants exactly L below are filled in.
// Iterative, depth-first, children in order 0, 1 (one frame per level,
// L <= kMaxL).
SC_HD void collect(const MaskInputs& b, int64_t m0, const float* gbox, const Grid& g,
                   uint32_t* out) {
  int64_t node[kMaxL];
  int depth[kMaxL], next[kMaxL];
  int sp = 0;
  node[0] = m0;
  depth[0] = 1;
  next[0] = 0;
  while (sp >= 0) {
    if (next[sp] == 2) {
      --sp;
      continue;
    }
    const int64_t m = node[sp];
    const int c = next[sp]++;
    const int32_t ch = b.child[2 * m + c], cn = b.count[2 * m + c];
    const float* cbox = &b.box[12 * m + 6 * c];
    if (depth[sp] == b.L) {
      fill_from_child(out, gbox, &b.masks[((size_t)m * 2 + c) * b.W], cbox, b.R, b.eps);
    } else if (cn > 0) {
      leaf_into(b, ch, cn, g, out);
    } else {
      node[sp + 1] = ch;
      depth[sp + 1] = depth[sp] + 1;
      next[sp + 1] = 0;
      ++sp;
    }
  }
}

// The mask of child slot c of node n (its deeper descendants' masks done).
SC_HD void slot_mask(const MaskInputs& b, int64_t n, int c) {
  uint32_t* out = &b.masks[((size_t)n * 2 + c) * b.W];
  const float* gbox = &b.box[12 * n + 6 * c];
  Grid g;
  g.init(gbox, b.R, b.eps);
  const int32_t ch = b.child[2 * n + c], cn = b.count[2 * n + c];
  if (cn > 0) leaf_into(b, ch, cn, g, out);
  else collect(b, ch, gbox, g, out);
}

}  // namespace mm
}  // namespace sc

#endif
