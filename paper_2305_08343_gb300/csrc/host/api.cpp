// api.cpp — host entry points of the C-ABI (include/subcull.h): inputs,
// build, export and image packing.  Device entry points live in
// cuda/trace.cu.  No exception leaves these functions.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>

#include "gen/scenegen.h"
#include "internal.h"

namespace sc {
const char* last_error_cstr();
}

using namespace sc;

#define SC_TRY                 \
  try {                        \
    clear_error();
#define SC_CATCH                                                  \
  }                                                               \
  catch (const Error& e) {                                        \
    set_error("%s", e.msg.c_str());                               \
    return e.code;                                                \
  }                                                               \
  catch (const std::bad_alloc&) {                                 \
    set_error("host allocation failed");                          \
    return SC_ERR_NOMEM;                                          \
  }                                                               \
  catch (...) {                                                   \
    set_error("unexpected internal error");                       \
    return SC_ERR_STATE;                                          \
  }

extern "C" {

const char* sc_last_error(void) { return last_error_cstr(); }
int sc_abi_version(void) { return SC_ABI_VERSION; }

sc_status sc_scene_generate(int kind, const sc_scene_params* p, uint64_t seed, float* tris,
                            int64_t cap, int64_t* n_tris) {
  SC_TRY
  if (!p || !n_tris) fail(SC_ERR_ARG, "sc_scene_generate: NULL params or n_tris");
  int64_t n;
  if (kind == SC_SCENE_HAIR) {
    if (p->count < 0 || p->segments < 1) fail(SC_ERR_ARG, "hair: bad strand/segment count");
    n = sg_hair_count(p->count, p->segments, p->ground);
  } else if (kind == SC_SCENE_SOUP) {
    if (p->count < 0) fail(SC_ERR_ARG, "soup: negative triangle count");
    n = p->count;
  } else {
    fail(SC_ERR_ARG, "unknown scene kind %d", kind);
  }
  *n_tris = n;
  if (!tris) return SC_OK;
  if (cap < n) fail(SC_ERR_NOMEM, "scene needs %lld triangles, buffer holds %lld", (long long)n,
                    (long long)cap);
  int T = resolve_threads(0);
  if (kind == SC_SCENE_HAIR) {
    parallel_ranges(p->count, T, [&](int64_t a, int64_t b, int) {
      sg_hair(seed, p->count, p->segments, 0, a, b, tris);
    });
    if (p->ground) sg_hair(seed, p->count, p->segments, 1, p->count, p->count, tris);
  } else {
    parallel_ranges(n, T, [&](int64_t a, int64_t b, int) { sg_soup(seed, a, b, tris); });
  }
  return SC_OK;
  SC_CATCH
}

sc_status sc_rays_generate(int kind, const sc_ray_params* p, uint64_t seed, float* rays,
                           int32_t* pix, int64_t cap, int64_t* n_rays) {
  SC_TRY
  if (!p || !n_rays) fail(SC_ERR_ARG, "sc_rays_generate: NULL params or n_rays");
  int64_t n;
  if (kind == SC_RAYS_PINHOLE) {
    if (p->width < 1 || p->height < 1) fail(SC_ERR_ARG, "pinhole: bad image size");
    n = (int64_t)p->width * p->height;
  } else if (kind == SC_RAYS_RANDOM) {
    if (p->count < 0) fail(SC_ERR_ARG, "random rays: negative count");
    n = p->count;
  } else {
    fail(SC_ERR_ARG, "unknown ray kind %d", kind);
  }
  *n_rays = n;
  if (!rays) return SC_OK;
  if (cap < n) fail(SC_ERR_NOMEM, "rays need %lld entries, buffer holds %lld", (long long)n,
                    (long long)cap);
  if (kind == SC_RAYS_PINHOLE) {
    sg_rays_pinhole(p->width, p->height, p->jitter_seed, rays, pix);
  } else {
    parallel_ranges(n, resolve_threads(0),
                    [&](int64_t a, int64_t b, int) { sg_rays_random(seed, a, b, rays); });
  }
  return SC_OK;
  SC_CATCH
}

void sc_build_opts_default(sc_build_opts* o) {
  if (!o) return;
  o->max_leaf = 4;
  o->bins = 32;
  o->L = 3;
  o->lut_size = 256;
  o->chunk_bits = 8;
  o->eps_rel = 1.0 / 65536.0;
  o->threads = 0;
  o->skip_bits = 0;
  o->test_stride = 1;
  o->leaf_min_tris = 0;
  o->gpu_masks = 0;
  o->gpu_bvh = 0;
}

sc_status sc_bvh_build(const float* tris, int64_t n, int grid_res, int compress,
                       const sc_build_opts* opts, sc_bvh** out) {
  SC_TRY
  if (!out) fail(SC_ERR_ARG, "sc_bvh_build: out is NULL");
  *out = nullptr;
  if (n < 0 || (n > 0 && !tris)) fail(SC_ERR_ARG, "sc_bvh_build: bad triangle array");
  if (n >= kMaxTris) fail(SC_ERR_UNSUPPORTED, "at most 2^28 - 1 triangles are supported");
  if (!(grid_res == 0 || grid_res == 4 || grid_res == 6 || grid_res == 8))
    fail(SC_ERR_UNSUPPORTED, "grid_res must be 0, 4, 6 or 8 (got %d)", grid_res);
  if (compress && grid_res == 0) fail(SC_ERR_ARG, "compression needs grid_res > 0");
  sc_build_opts o;
  sc_build_opts_default(&o);
  if (opts) o = *opts;
  if (o.max_leaf < 1 || o.max_leaf > kMaxLeafTris) fail(SC_ERR_ARG, "max_leaf must be 1..8");
  if (o.bins < 2 || o.bins > 256) fail(SC_ERR_ARG, "bins must be 2..256");
  if (o.L < 1) fail(SC_ERR_ARG, "L must be >= 1");
  if (o.lut_size < 1 || o.lut_size > 256) fail(SC_ERR_ARG, "lut_size must be 1..256");
  if (o.chunk_bits < 1 || o.chunk_bits > 12) fail(SC_ERR_ARG, "chunk_bits must be 1..12");
  if (!(o.eps_rel >= 0.0)) fail(SC_ERR_ARG, "eps_rel must be >= 0");
  if (o.skip_bits < 0) fail(SC_ERR_ARG, "skip_bits must be >= 0");
  if (o.test_stride < 0) fail(SC_ERR_ARG, "test_stride must be >= 0");
  if (o.leaf_min_tris < 0) fail(SC_ERR_ARG, "leaf_min_tris must be >= 0");
  if (o.gpu_bvh && o.bins > 32)
    fail(SC_ERR_UNSUPPORTED, "the GPU tree builder takes at most 32 bins (got %d)", o.bins);
  for (int64_t i = 0; i < 9 * n; ++i)
    if (!std::isfinite(tris[i])) fail(SC_ERR_ARG, "triangle %lld has a non-finite coordinate",
                                      (long long)(i / 9));
  int T = resolve_threads(o.threads);
  sc_bvh* h = new sc_bvh();
  try {
    h->b.opts = o;
    if (o.gpu_bvh)
      build_bvh_gpu(h->b, tris, n, o.max_leaf, o.bins);
    else
      build_bvh(h->b, tris, n, o.max_leaf, o.bins, T);
    if (grid_res > 0) {
      if (o.gpu_masks)
        build_masks_gpu(h->b, grid_res, o.L, scene_eps(tris, n, o.eps_rel));
      else
        build_masks(h->b, grid_res, o.L, scene_eps(tris, n, o.eps_rel), T);
      if (compress) build_compression(h->b, o.lut_size, o.chunk_bits, T);
    }
  } catch (...) {
    delete h;
    throw;
  }
  *out = h;
  return SC_OK;
  SC_CATCH
}

void sc_bvh_destroy(sc_bvh* b) { delete b; }

sc_status sc_bvh_get_info(const sc_bvh* h, sc_bvh_info* info) {
  SC_TRY
  if (!h || !info) fail(SC_ERR_ARG, "sc_bvh_get_info: NULL argument");
  const Bvh& b = h->b;
  std::memset(info, 0, sizeof(*info));
  info->num_tris = b.ntri;
  info->num_nodes = b.nn;
  info->max_depth = b.max_depth;
  info->grid_res = b.R;
  info->compress = b.compress;
  info->L = b.L;
  info->clut_entries = b.K;
  info->eps = b.eps;
  std::memcpy(info->root_box, b.root_box, sizeof(info->root_box));
  info->ms_bvh = b.ms_bvh;
  info->ms_masks = b.ms_masks;
  info->ms_compress = b.ms_compress;
  return SC_OK;
  SC_CATCH
}

sc_status sc_bvh_export(const sc_bvh* h, int32_t* root2, int32_t* child, int32_t* count,
                        float* box, int32_t* perm, uint32_t* masks, uint32_t* clut,
                        uint8_t* cidx) {
  SC_TRY
  if (!h) fail(SC_ERR_ARG, "sc_bvh_export: NULL bvh");
  const Bvh& b = h->b;
  if (root2) {
    root2[0] = b.root_child;
    root2[1] = b.root_count;
  }
  if (child) std::memcpy(child, b.child.data(), 4 * b.child.size());
  if (count) std::memcpy(count, b.count.data(), 4 * b.count.size());
  if (box) std::memcpy(box, b.box.data(), 4 * b.box.size());
  if (perm) std::memcpy(perm, b.perm.data(), 4 * b.perm.size());
  if (masks) {
    if (b.R == 0) fail(SC_ERR_STATE, "BVH was built without masks");
    std::memcpy(masks, b.masks.data(), 4 * b.masks.size());
  }
  if (clut || cidx) {
    if (!b.compress) fail(SC_ERR_STATE, "BVH was built without compression");
    if (clut) std::memcpy(clut, b.clut.data(), 4 * b.clut.size());
    if (cidx) std::memcpy(cidx, b.cidx.data(), b.cidx.size());
  }
  return SC_OK;
  SC_CATCH
}

sc_status sc_bvh_frontier(const sc_bvh* h, int depth, sc_frontier_entry* out, int cap,
                          int* n_slots, uint8_t* class_of_tri) {
  SC_TRY
  if (!h || !out || !n_slots || depth < 0 || depth > 8 || cap < 1)
    fail(SC_ERR_ARG, "sc_bvh_frontier: bad argument (depth 0..8)");
  const Bvh& b = h->b;
  int n = 0;
  *n_slots = 0;
  if (b.ntri == 0) return SC_OK;
  struct It {
    int32_t child, count;
    int depth;
    const float* box;
  };
  std::vector<It> st;
  st.push_back(It{b.root_child, b.root_count, 0, b.root_box});
  while (!st.empty()) {
    It it = st.back();
    st.pop_back();
    if (it.count > 0 || it.depth == depth) {
      if (n >= cap) fail(SC_ERR_NOMEM, "sc_bvh_frontier: more than %d slots", cap);
      sc_frontier_entry& e = out[n];
      std::memcpy(e.lo, it.box, 3 * sizeof(float));
      std::memcpy(e.hi, it.box + 3, 3 * sizeof(float));
      e.slot = it.count > 0 ? (kLeafBit | ((uint32_t)(it.count - 1) << 28) | (uint32_t)it.child)
                            : (uint32_t)it.child;
      e.reserved = 0;
      if (class_of_tri) {
        // the triangle positions of a subtree form one contiguous range
        int64_t lo = INT64_MAX, hi = -1;
        std::vector<It> sub{it};
        while (!sub.empty()) {
          It x = sub.back();
          sub.pop_back();
          if (x.count > 0) {
            lo = std::min<int64_t>(lo, x.child);
            hi = std::max<int64_t>(hi, (int64_t)x.child + x.count);
          } else {
            for (int c = 0; c < 2; ++c)
              sub.push_back(It{b.child[2 * x.child + c], b.count[2 * x.child + c], 0, nullptr});
          }
        }
        for (int64_t pos = lo; pos < hi; ++pos) class_of_tri[b.perm[pos]] = (uint8_t)n;
      }
      ++n;
      continue;
    }
    // push the right child first: pre-order visits the left subtree first
    for (int c = 1; c >= 0; --c)
      st.push_back(It{b.child[2 * it.child + c], b.count[2 * it.child + c], it.depth + 1,
                      &b.box[12 * (size_t)it.child + 6 * c]});
  }
  *n_slots = n;
  return SC_OK;
  SC_CATCH
}

sc_status sc_raylut(int R, uint32_t* lut) {
  SC_TRY
  if (!(R == 2 || R == 3 || R == 4 || R == 6 || R == 8) || !lut)
    fail(SC_ERR_ARG, "sc_raylut: R must be 2, 3, 4, 6 or 8 and lut non-NULL");
  raylut_full(R, lut);
  return SC_OK;
  SC_CATCH
}

sc_status sc_raylut2r(int R, uint32_t* lut) {
  SC_TRY
  if (!(R == 2 || R == 3 || R == 4 || R == 6) || !lut)
    fail(SC_ERR_ARG, "sc_raylut2r: R must be 2, 3, 4 or 6 and lut non-NULL");
  raylut2r_full(R, lut);
  return SC_OK;
  SC_CATCH
}

sc_status sc_bvh_device_bytes(const sc_bvh* h, int layout, size_t* nbytes) {
  SC_TRY
  if (!h || !nbytes) fail(SC_ERR_ARG, "sc_bvh_device_bytes: NULL argument");
  *nbytes = image_layout(h->b, layout).total;
  return SC_OK;
  SC_CATCH
}

}  // extern "C"
