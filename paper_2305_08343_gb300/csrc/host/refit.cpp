// refit.cpp — updating a built BVH for moved triangles (dynamic scenes; the
// paper leaves efficient mask updates for animated primitives to future
// work).
//
// The tree's topology and triangle order are kept.  A triangle has moved
// when any of its nine coordinates differs bit for bit from the stored one.
// Boxes are refit bottom-up: a leaf slot's box is the union of its
// triangles' boxes, an inner slot's the union of its child node's two slot
// boxes -- the same union over the same triangles that the build takes, so
// an unmoved subtree keeps its box exactly.  A node is dirty when a moved
// triangle lies below either of its slots; only dirty nodes' masks are
// computed again (a slot's mask depends only on its box and what lies below
// it), on the host or the GPU as the build chose, and for compressed BVHs
// only their slots are encoded again (Alg. 3) against the LUT chosen at
// build time.  If the scene's dilation eps (relative to the largest
// coordinate) changes, every node is dirty.  The result equals a mask build
// from scratch on the refit tree.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "internal.h"

using namespace sc;

namespace {

inline void tri_box(const float* t, float* lo, float* hi) {
  for (int k = 0; k < 3; ++k) {
    lo[k] = std::fmin(std::fmin(t[k], t[3 + k]), t[6 + k]);
    hi[k] = std::fmax(std::fmax(t[k], t[3 + k]), t[6 + k]);
  }
}

inline void box_empty(float* b) {
  b[0] = b[1] = b[2] = INFINITY;
  b[3] = b[4] = b[5] = -INFINITY;
}

inline void box_grow(float* b, const float* lo, const float* hi) {
  for (int k = 0; k < 3; ++k) {
    b[k] = std::fmin(b[k], lo[k]);
    b[3 + k] = std::fmax(b[3 + k], hi[k]);
  }
}

// If a triangle at leaf positions [first, first + count) moved: its box,
// and true.
bool leaf_box(const Bvh& b, const std::vector<uint8_t>& moved, int32_t first, int32_t count,
              float* box) {
  bool dirty = false;
  for (int32_t i = 0; i < count; ++i) dirty |= moved[b.perm[first + i]] != 0;
  if (!dirty) return false;
  box_empty(box);
  for (int32_t i = 0; i < count; ++i) {
    float lo[3], hi[3];
    tri_box(&b.tris[9 * (size_t)b.perm[first + i]], lo, hi);
    box_grow(box, lo, hi);
  }
  return true;
}

}  // namespace

#define SC_TRY \
  try {        \
    clear_error();
#define SC_CATCH                           \
  }                                        \
  catch (const Error& e) {                 \
    set_error("%s", e.msg.c_str());        \
    return e.code;                         \
  }                                        \
  catch (const std::bad_alloc&) {          \
    set_error("host allocation failed");   \
    return SC_ERR_NOMEM;                   \
  }                                        \
  catch (...) {                            \
    set_error("unexpected internal error"); \
    return SC_ERR_STATE;                   \
  }

extern "C" {

sc_status sc_bvh_refit(sc_bvh* h, const float* tris, int64_t n_tris, sc_refit_info* info) {
  SC_TRY
  if (!h) fail(SC_ERR_ARG, "sc_bvh_refit: NULL bvh");
  Bvh& b = h->b;
  if (n_tris != b.ntri)
    fail(SC_ERR_ARG, "sc_bvh_refit: %lld triangles, the BVH holds %lld", (long long)n_tris,
         (long long)b.ntri);
  if (n_tris > 0 && !tris) fail(SC_ERR_ARG, "sc_bvh_refit: NULL triangles");
  for (int64_t i = 0; i < 9 * n_tris; ++i)
    if (!std::isfinite(tris[i]))
      fail(SC_ERR_ARG, "triangle %lld has a non-finite coordinate", (long long)(i / 9));
  const double t0 = now_ms();
  const int T = resolve_threads(b.opts.threads);
  // moved triangles (copied in), and the largest coordinate for eps
  std::vector<uint8_t> moved((size_t)n_tris, 0);
  const int parts = std::max(1, std::min<int>(T, (int)(n_tris / 65536) + 1));
  std::vector<int64_t> part_moved(parts, 0);
  std::vector<double> part_max(parts, 1.0);
  parallel_ranges(n_tris, parts, [&](int64_t lo, int64_t hi, int p) {
    int64_t m = 0;
    double s = 1.0;
    for (int64_t i = lo; i < hi; ++i) {
      float* old = &b.tris[9 * (size_t)i];
      const float* nw = tris + 9 * i;
      if (std::memcmp(old, nw, 9 * sizeof(float)) != 0) {
        std::memcpy(old, nw, 9 * sizeof(float));
        moved[i] = 1;
        ++m;
      }
      for (int k = 0; k < 9; ++k) {
        const double a = std::fabs((double)nw[k]);
        if (a > s) s = a;
      }
    }
    part_moved[p] = m;
    part_max[p] = s;
  });
  int64_t n_moved = 0;
  double max_abs = 1.0;
  for (int p = 0; p < parts; ++p) {
    n_moved += part_moved[p];
    max_abs = std::max(max_abs, part_max[p]);
  }
  // boxes bottom-up: children are numbered after their parents
  std::vector<uint8_t> dirty((size_t)b.nn, 0);
  for (int64_t n = b.nn - 1; n >= 0 && n_moved; --n) {
    bool d = false;
    for (int c = 0; c < 2; ++c) {
      float* box = &b.box[12 * (size_t)n + 6 * c];
      const int32_t ch = b.child[2 * n + c], cn = b.count[2 * n + c];
      if (cn > 0) {
        float nb[6];
        if (leaf_box(b, moved, ch, cn, nb)) {
          std::memcpy(box, nb, sizeof(nb));
          d = true;
        }
      } else if (dirty[ch]) {
        box_empty(box);
        box_grow(box, &b.box[12 * (size_t)ch], &b.box[12 * (size_t)ch + 3]);
        box_grow(box, &b.box[12 * (size_t)ch + 6], &b.box[12 * (size_t)ch + 9]);
        d = true;
      }
    }
    dirty[n] = d;
  }
  if (n_moved && b.ntri > 0) {
    if (b.root_count > 0) {
      leaf_box(b, moved, b.root_child, b.root_count, b.root_box);
    } else {
      box_empty(b.root_box);
      box_grow(b.root_box, &b.box[0], &b.box[3]);
      box_grow(b.root_box, &b.box[6], &b.box[9]);
    }
  }
  const double t1 = now_ms();
  int64_t n_dirty = 0;
  for (uint8_t d : dirty) n_dirty += d;
  double ms_masks = 0.0, ms_compress = 0.0;
  if (b.R > 0 && n_moved) {
    const double eps = b.opts.eps_rel * max_abs;  // scene_eps of the moved scene
    if (eps != b.eps) {
      b.eps = eps;
      std::fill(dirty.begin(), dirty.end(), 1);
      n_dirty = b.nn;
    }
    const double build_ms = b.ms_masks;  // the build's figure stays in the handle
    if (b.opts.gpu_masks)
      refit_masks_gpu(b, dirty);
    else
      refit_masks(b, dirty, T);
    ms_masks = b.ms_masks;
    b.ms_masks = build_ms;
    if (b.compress) {
      const double t2 = now_ms();
      encode_slots(b, T, &dirty);
      ms_compress = now_ms() - t2;
    }
  }
  if (info) {
    info->moved_tris = n_moved;
    info->dirty_nodes = n_dirty;
    info->ms_boxes = t1 - t0;
    info->ms_masks = ms_masks;
    info->ms_compress = ms_compress;
  }
  return SC_OK;
  SC_CATCH
}

}  // extern "C"
