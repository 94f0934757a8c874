// masks.cpp — object masks of every child slot of the BVH2.
//
//  * Leaf slot: conservative voxelization of its triangles (Sec. 3.1.1) in
//    the slot box's R^3 grid — a voxel is set iff the triangle overlaps the
//    voxel box dilated by eps (separating-axis test, double precision).
//  * Inner slot (Sec. 3.2.1, parameter L): OR of the direct voxelization of
//    the triangles of every leaf fewer than L levels below the slot's node,
//    and of Alg. 2 (fill by approximated occupancy) applied to the mask of
//    every descendant exactly L levels below.  With borders dilated by eps,
//    Alg. 2 keeps "every cell within eps of a triangle is set".
//  * Slots are processed level by level from the deepest, so each level
//    reads only finished masks of deeper nodes; a level is parallel.
// The voxel bounds, the 13-axis test and the fill indices are evaluated with
// exactly the operation sequence of their definitions below, so that any
// implementation of the same definitions sets the same bits.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace sc {
namespace {

inline double mn(double a, double b) { return a < b ? a : b; }
inline double mx(double a, double b) { return a > b ? a : b; }

// Separating-axis triangle/box overlap (Akenine-Moeller 2001); touching
// counts as overlap.  v: 9 doubles.
bool tri_box_overlap(const double* v, const double* bmin, const double* bmax) {
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
  const double rn = (h[0] * std::fabs(nx) + h[1] * std::fabs(ny)) + h[2] * std::fabs(nz);
  if (std::fabs(d) > rn) return false;
  for (int i = 0; i < 3; ++i) {
    const double ex = e[i][0], ey = e[i][1], ez = e[i][2];
    const double axes[3][3] = {{0.0, ez, -ey}, {-ez, 0.0, ex}, {ey, -ex, 0.0}};
    for (int k = 0; k < 3; ++k) {
      const double* ax = axes[k];
      double p0 = (ax[0] * a[0][0] + ax[1] * a[0][1]) + ax[2] * a[0][2];
      double p1 = (ax[0] * a[1][0] + ax[1] * a[1][1]) + ax[2] * a[1][2];
      double p2 = (ax[0] * a[2][0] + ax[1] * a[2][1]) + ax[2] * a[2][2];
      double r = (h[0] * std::fabs(ax[0]) + h[1] * std::fabs(ax[1])) + h[2] * std::fabs(ax[2]);
      if (mn(mn(p0, p1), p2) > r || mx(mx(p0, p1), p2) < -r) return false;
    }
  }
  return true;
}

// Grid of one slot: per axis the dilated voxel bounds.
struct Grid {
  int R;
  double eps;
  double lo[3], ext[3];
  double b0[3][16], b1[3][16];
  void init(const float* box, int R_, double eps_) {
    R = R_;
    eps = eps_;
    for (int k = 0; k < 3; ++k) {
      lo[k] = (double)box[k];
      ext[k] = (double)box[3 + k] - (double)box[k];
      for (int i = 0; i < R; ++i) {
        b0[k][i] = (lo[k] + (ext[k] * (double)i) / (double)R) - eps_;
        b1[k][i] = (lo[k] + (ext[k] * (double)(i + 1)) / (double)R) + eps_;
      }
    }
  }
  // Voxels [i0, i1] on axis k whose dilated box may overlap [tlo, thi]; one
  // voxel of margin beyond the eps-widened range keeps this a superset of
  // what the exact test keeps.
  void candidates(int k, double tlo, double thi, int& i0, int& i1) const {
    double w = ext[k] / (double)R;
    if (!(w > 1e-12 * mx(1.0, std::fabs(lo[k])))) {
      i0 = 0;
      i1 = R - 1;
      return;
    }
    double q0 = std::floor(((tlo - eps) - lo[k]) / w) - 1.0;
    double q1 = std::floor(((thi + eps) - lo[k]) / w) + 1.0;
    q0 = mx(0.0, mn(q0, (double)(R - 1)));
    q1 = mx(0.0, mn(q1, (double)(R - 1)));
    i0 = (int)q0;
    i1 = (int)q1;
  }
};

inline void set_bit(uint32_t* m, int bit) { m[bit >> 5] |= 1u << (bit & 31); }
inline bool get_bit(const uint32_t* m, int bit) { return (m[bit >> 5] >> (bit & 31)) & 1u; }

void voxelize_tri(const float* t9, const Grid& g, uint32_t* out) {
  double v[9];
  for (int i = 0; i < 9; ++i) v[i] = (double)t9[i];
  int r0[3], r1[3];
  for (int k = 0; k < 3; ++k) {
    double tlo = mn(mn(v[k], v[3 + k]), v[6 + k]);
    double thi = mx(mx(v[k], v[3 + k]), v[6 + k]);
    g.candidates(k, tlo, thi, r0[k], r1[k]);
  }
  const int R = g.R;
  for (int z = r0[2]; z <= r1[2]; ++z)
    for (int y = r0[1]; y <= r1[1]; ++y)
      for (int x = r0[0]; x <= r1[0]; ++x) {
        int bit = x + R * y + R * R * z;
        if (get_bit(out, bit)) continue;
        double bmin[3] = {g.b0[0][x], g.b0[1][y], g.b0[2][z]};
        double bmax[3] = {g.b1[0][x], g.b1[1][y], g.b1[2][z]};
        if (tri_box_overlap(v, bmin, bmax)) set_bit(out, bit);
      }
}

// Alg. 2 parent index: min(floor(R * (pos - pLower) / pExtent), R-1), >= 0.
inline int parent_idx(double pos, double plo, double pext, int R) {
  double q = std::floor(((double)R * (pos - plo)) / pext);
  q = q < 0.0 ? 0.0 : q;
  q = q > (double)(R - 1) ? (double)(R - 1) : q;
  return (int)q;
}

// Alg. 2 (fillByApproximatedOccupancy) with borders dilated by eps.
void fill_from_child(uint32_t* out, const float* pbox, const uint32_t* cmask,
                     const float* cbox, int R, double eps) {
  int lo_i[3][17], hi_i[3][17];
  for (int k = 0; k < 3; ++k) {
    double cl = (double)cbox[k], cext = (double)cbox[3 + k] - (double)cbox[k];
    double pl = (double)pbox[k], pext = (double)pbox[3 + k] - (double)pbox[k];
    for (int i = 0; i <= R; ++i) {
      double border = cl + (cext * (double)i) / (double)R;
      if (pext > 0.0) {
        lo_i[k][i] = parent_idx(border - eps, pl, pext, R);
        hi_i[k][i] = parent_idx(border + eps, pl, pext, R);
      } else {
        lo_i[k][i] = 0;
        hi_i[k][i] = R - 1;
      }
    }
  }
  // per-axis range masks, combined as a box pattern
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

struct MaskBuilder {
  Bvh& b;
  void leaf_into(int32_t first, int32_t count, const Grid& g, uint32_t* out) const {
    for (int32_t i = 0; i < count; ++i)
      voxelize_tri(&b.tris[9 * (size_t)b.perm[first + i]], g, out);
  }
  void collect(int64_t m, int depth, const float* gbox, const Grid& g, uint32_t* out) const {
    for (int c = 0; c < 2; ++c) {
      int32_t ch = b.child[2 * m + c], cn = b.count[2 * m + c];
      const float* cbox = &b.box[12 * m + 6 * c];
      if (depth == b.L) {
        fill_from_child(out, gbox, &b.masks[((size_t)m * 2 + c) * b.W], cbox, b.R, b.eps);
      } else if (cn > 0) {
        leaf_into(ch, cn, g, out);
      } else {
        collect(ch, depth + 1, gbox, g, out);
      }
    }
  }
  void slot(int64_t n, int c) const {
    uint32_t* out = &b.masks[((size_t)n * 2 + c) * b.W];
    const float* gbox = &b.box[12 * n + 6 * c];
    Grid g;
    g.init(gbox, b.R, b.eps);
    int32_t ch = b.child[2 * n + c], cn = b.count[2 * n + c];
    if (cn > 0) leaf_into(ch, cn, g, out);
    else collect(ch, 1, gbox, g, out);
  }
};

}  // namespace

void build_masks(Bvh& b, int R, int L, double eps, int threads) {
  double t0 = now_ms();
  b.R = R;
  b.L = L;
  b.W = mask_words(R);
  b.eps = eps;
  b.masks.assign((size_t)b.nn * 2 * b.W, 0u);
  // nodes grouped by depth, deepest level first
  std::vector<std::vector<int64_t>> levels(b.max_depth + 1);
  for (int64_t n = 0; n < b.nn; ++n) levels[b.ndepth[n]].push_back(n);
  MaskBuilder mb{b};
  for (int d = b.max_depth; d >= 0; --d) {
    const auto& lv = levels[d];
    parallel_for((int64_t)lv.size() * 2, threads, 256, [&](int64_t i) {
      mb.slot(lv[i >> 1], (int)(i & 1));
    });
  }
  b.ms_masks = now_ms() - t0;
}

}  // namespace sc
