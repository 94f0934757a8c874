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
#include "mask_math.h"

namespace sc {

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
  // levels below the tree's depth change nothing: L is used up to max_depth + 1
  if (std::min(L, b.max_depth + 1) > mm::kMaxL)
    fail(SC_ERR_UNSUPPORTED, "mask depth L = %d over a tree %d deep exceeds %d", L,
         b.max_depth, mm::kMaxL);
  const mm::MaskInputs in{b.tris.data(), b.perm.data(), b.child.data(), b.count.data(),
                          b.box.data(),      b.masks.data(), R, std::min(L, b.max_depth + 1),
                          b.W,               eps};
  for (int d = b.max_depth; d >= 0; --d) {
    const auto& lv = levels[d];
    parallel_for((int64_t)lv.size() * 2, threads, 256, [&](int64_t i) {
      mm::slot_mask(in, lv[i >> 1], (int)(i & 1));
    });
  }
  b.ms_masks = now_ms() - t0;
}

// Masks of the nodes marked in node_dirty only (both slots of each), deepest
// level first; every other mask is kept.  A slot's mask depends only on its
// box and what lies below it, so after a refit only slots above a moved
// triangle need it again.
void refit_masks(Bvh& b, const std::vector<uint8_t>& node_dirty, int threads) {
  double t0 = now_ms();
  std::vector<std::vector<int64_t>> levels(b.max_depth + 1);
  for (int64_t n = 0; n < b.nn; ++n)
    if (node_dirty[n]) levels[b.ndepth[n]].push_back(n);
  const mm::MaskInputs in{b.tris.data(), b.perm.data(), b.child.data(), b.count.data(),
                          b.box.data(),      b.masks.data(), b.R, std::min(b.L, b.max_depth + 1),
                          b.W,               b.eps};
  for (int d = b.max_depth; d >= 0; --d) {
    const auto& lv = levels[d];
    parallel_for((int64_t)lv.size() * 2, threads, 256, [&](int64_t i) {
      const int64_t n = lv[i >> 1];
      const int c = (int)(i & 1);
      std::memset(&b.masks[((size_t)n * 2 + c) * b.W], 0, sizeof(uint32_t) * b.W);
      mm::slot_mask(in, n, c);
    });
  }
  b.ms_masks = now_ms() - t0;
}

}  // namespace sc
