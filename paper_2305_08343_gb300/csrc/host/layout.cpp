// layout.cpp — the device image of a BVH (node records, triangles, tables).
//
// Nodes are child pairs of 64 bytes (four 16-byte vectors, one 128-bit load
// each): {lo0.x, lo0.y, hi0.x, hi0.y} {lo1.x, lo1.y, hi1.x, hi1.y}
// {lo0.z, hi0.z, lo1.z, hi1.z} {slot0, slot1, meta0, meta1}, so that each
// child's x, y bounds are adjacent for packed two-lane arithmetic.  The
// masked layout adds the two children's Alg. 1 scales
// R / extent (32 bytes) and, uncompressed, the two R^3-bit object masks
// (mask_stride bytes each, zero padded): 128 / 160 / 224 bytes at
// R = 4 / 6 / 8 (records are padded to whole 32-byte sectors), the scales as
// {s0.x, s0.y, s1.x, s1.y} {s0.z, s1.z, 0, 0}; compressed, the 1-byte LUT
// index of each child sits in the
// fourth vector (Sec. 3.2.4: the index replaces the mask) and the node is
// 96 bytes.  The compact masked layout omits the scales (96 / 128 / 192 and
// 64 bytes).  Records stay 32-byte aligned: the masks are compared with
// 256-bit loads.
// Triangles are 48 bytes in leaf order: {v0, id}, {e1 = v1 - v0}, {e2 =
// v2 - v0}.  Every region starts on a 256-byte boundary.
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace sc {

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// A child is kept without a test when its mask has >= skip bits set (an
// all-ones mask can never be culled; denser masks rarely are).
static bool skip_test(const uint32_t* m, int R, int skip_bits) {
  const int R3 = R * R * R;
  int pop = 0;
  for (int w = 0; w < (R3 + 31) / 32; ++w) pop += __builtin_popcount(m[w]);
  return pop >= (skip_bits > 0 ? skip_bits : R3);
}

uint32_t root_slot_word(const Bvh& b) {
  if (b.root_count > 0)
    return kLeafBit | ((uint32_t)(b.root_count - 1) << 28) | (uint32_t)b.root_child;
  return 0u;
}

static uint32_t slot_word(int32_t child, int32_t count) {
  if (count > 0) return kLeafBit | ((uint32_t)(count - 1) << 28) | (uint32_t)child;
  return (uint32_t)child;
}

// 4-wide view: the node made from binary node n takes, in order, for each
// child slot c of n, the two child slots of c if c is inner, else c itself;
// inner children are the nodes made from their binary nodes; pre-order.
struct Wide {
  std::vector<int32_t> n;     // [nodes] children (2..4)
  std::vector<int64_t> p;     // [nodes][4] binary parent of each child slot
  std::vector<int32_t> c;     // [nodes][4] child index in that parent
  std::vector<int64_t> next;  // [nodes][4] wide node of an inner child, -1 leaf
  int depth = 0;
};

static void wide_build(const Bvh& b, Wide& w) {
  if (b.ntri == 0 || b.root_count > 0) return;
  struct Item {
    int64_t n;       // binary node the wide node is made from
    int depth;
    int64_t parent;  // wide parent (-1: the root) and its child index
    int slot;
  };
  // pre-order: a node, then the whole subtree of its first inner child,
  // then the next (a stack with the children pushed in reverse)
  std::vector<Item> st{Item{b.root_child, 0, -1, 0}};
  while (!st.empty()) {
    const Item it = st.back();
    st.pop_back();
    const int64_t q = (int64_t)w.n.size();
    if (it.parent >= 0) w.next[4 * it.parent + it.slot] = q;
    w.depth = std::max(w.depth, it.depth);
    w.n.push_back(0);
    for (int k = 0; k < 4; ++k) {
      w.p.push_back(-1);
      w.c.push_back(0);
      w.next.push_back(-1);
    }
    int k = 0;
    for (int c = 0; c < 2; ++c) {
      if (b.count[2 * it.n + c] == 0) {
        const int64_t m = b.child[2 * it.n + c];
        for (int g = 0; g < 2; ++g, ++k) {
          w.p[4 * q + k] = m;
          w.c[4 * q + k] = g;
        }
      } else {
        w.p[4 * q + k] = it.n;
        w.c[4 * q + k] = c;
        ++k;
      }
    }
    w.n[q] = k;
    for (int i = k - 1; i >= 0; --i) {
      const int64_t pp = w.p[4 * q + i];
      const int cc = w.c[4 * q + i];
      if (b.count[2 * pp + cc] == 0) st.push_back(Item{b.child[2 * pp + cc], it.depth + 1, q, i});
    }
  }
}

ImageLayout image_layout(const Bvh& b, int layout) {
  ImageLayout L;
  L.layout = layout;
  if (layout == SC_LAYOUT_PLAIN4 || layout == SC_LAYOUT_MASKED4) {
    Wide w;
    wide_build(b, w);
    L.width = 4;
    L.nodes = (int64_t)w.n.size();
    L.stack_need = 3 * (w.depth + 1) + 1;
    L.node_bytes = 128;
    if (layout == SC_LAYOUT_MASKED4) {
      if (b.R <= 0) fail(SC_ERR_STATE, "masked layout requested for a BVH built without masks");
      L.R = b.R;
      L.W = mask_words(b.R);
      L.mstride = mask_stride(b.R);
      L.compress = b.compress;
      L.K = b.K;
      L.scales = 1;
      // the masks start on a 32-byte boundary (16 bytes of padding after
      // the scales): they are compared with 256-bit loads
      L.mask_off = 192;
      L.node_bytes = b.compress ? 176 : 192 + 4 * L.mstride;
    }
  } else {
    L.nodes = b.nn;
    L.stack_need = b.max_depth + 1;
  }
  if (layout == SC_LAYOUT_MASKED || layout == SC_LAYOUT_MASKED_COMPACT ||
      layout == SC_LAYOUT_MASKED_RAY2R) {
    if (b.R <= 0) fail(SC_ERR_STATE, "masked layout requested for a BVH built without masks");
    if (layout == SC_LAYOUT_MASKED_RAY2R && (b.compress || b.R > 6))
      fail(SC_ERR_UNSUPPORTED,
           "the R_ray = 2R table needs uncompressed masks and R = 4 or 6 (R = %d%s)", b.R,
           b.compress ? ", compressed" : "");
    L.R = b.R;
    L.W = mask_words(b.R);
    L.mstride = mask_stride(b.R);
    L.compress = b.compress;
    L.K = b.K;
    L.scales = layout == SC_LAYOUT_MASKED_COMPACT ? 0 : 1;
    L.ray2r = layout == SC_LAYOUT_MASKED_RAY2R ? 1 : 0;
    L.mask_off = L.scales ? 96 : 64;
    L.node_bytes = b.compress ? L.mask_off : L.mask_off + 2 * L.mstride;
    // whole 32-byte sectors: the kernels compare the masks with 256-bit
    // loads, which need 32-byte aligned addresses
    L.node_bytes = (L.node_bytes + 31) / 32 * 32;
  } else if (layout != SC_LAYOUT_PLAIN && layout != SC_LAYOUT_PLAIN4 &&
             layout != SC_LAYOUT_MASKED4) {
    fail(SC_ERR_ARG, "unknown layout %d", layout);
  }
  size_t off = 256;
  L.off_nodes = off;
  off = align256(off + (size_t)L.nodes * L.node_bytes);
  L.off_tris = off;
  off = align256(off + (size_t)b.ntri * 48);
  if (L.R > 0) {
    size_t R3 = (size_t)L.R * L.R * L.R;
    L.off_lut = off;
    off = align256(off + R3 * R3 * L.mstride);
    L.off_pair = off;
    off = align256(off + R3 * L.R * 8);
    if (L.compress) {
      L.off_clut = off;
      off = align256(off + (size_t)256 * L.mstride);
      L.off_bits = off;
      off = align256(off + R3 * R3 * 32);
    }
    if (L.ray2r) {
      const size_t R23 = (size_t)8 * R3;
      L.off_lut2 = off;
      off = align256(off + R23 * R23 * L.mstride);
    }
  }
  L.total = off;
  return L;
}

namespace {
// The R_ray = 2R table depends on R alone (about a second to build at R = 6):
// built once per R and kept.
const std::vector<uint32_t>& raylut2r_cached(int R) {
  static std::mutex mu;
  static std::vector<uint32_t> tables[9];
  std::lock_guard<std::mutex> lock(mu);
  std::vector<uint32_t>& t = tables[R];
  if (t.empty()) {
    const size_t R23 = (size_t)8 * R * R * R;
    t.assign(R23 * R23 * mask_words(R), 0u);
    raylut2r_full(R, t.data());
  }
  return t;
}
}  // namespace

void pack_image(const Bvh& b, const ImageLayout& L, std::vector<uint8_t>& img) {
  img.assign(L.total, 0);
  uint8_t* base = img.data();
  // header: a few words for debugging tools
  uint32_t* hdr = reinterpret_cast<uint32_t*>(base);
  hdr[0] = 0x4C554353u;  // "SCUL"
  hdr[1] = SC_ABI_VERSION;
  hdr[2] = (uint32_t)L.layout;
  hdr[3] = (uint32_t)L.R;
  hdr[4] = (uint32_t)b.nn;
  hdr[5] = (uint32_t)b.ntri;
  hdr[6] = root_slot_word(b);
  // meta word of binary child slot (n, c): LUT index and "keep untested"
  auto meta_of = [&](int64_t n, int c) -> uint32_t {
    const uint32_t* m = L.compress ? &b.clut[(size_t)b.cidx[2 * n + c] * L.W]
                                   : &b.masks[((size_t)n * 2 + c) * L.W];
    uint32_t meta = L.compress ? (uint32_t)b.cidx[2 * n + c] : 0u;
    const int stride = b.opts.test_stride > 1 ? b.opts.test_stride : 1;
    const int32_t cnt = b.count[2 * n + c];
    const bool inner = cnt == 0;
    if (skip_test(m, L.R, b.opts.skip_bits) || (inner && (b.ndepth[n] + 1) % stride != 0) ||
        (!inner && cnt < b.opts.leaf_min_tris))
      meta |= kMetaFull;
    return meta;
  };
  if (L.width == 4) {
    Wide w;
    wide_build(b, w);
    parallel_for((int64_t)w.n.size(), resolve_threads(0), 8192, [&](int64_t q) {
      uint8_t* rec = base + L.off_nodes + (size_t)q * L.node_bytes;
      float* f = reinterpret_cast<float*>(rec);
      uint32_t* slots = reinterpret_cast<uint32_t*>(rec + 96);
      uint32_t* metas = reinterpret_cast<uint32_t*>(rec + 112);
      for (int i = 0; i < 4; ++i) {
        if (i >= w.n[q]) {
          for (int k = 0; k < 3; ++k) {
            f[4 * k + i] = 1.0f;       // an empty box (lo > hi); never tested:
            f[4 * (3 + k) + i] = 0.0f;  // the slot word marks the child unused
          }
          slots[i] = 0xFFFFFFFFu;
          metas[i] = kMetaFull;
          if (L.scales)
            for (int k = 0; k < 3; ++k) reinterpret_cast<float*>(rec + 128)[4 * k + i] = 0.0f;
          continue;
        }
        const int64_t pn = w.p[4 * q + i];
        const int c = w.c[4 * q + i];
        const float* bx = &b.box[12 * pn + 6 * c];
        for (int k = 0; k < 3; ++k) {
          f[4 * k + i] = bx[k];
          f[4 * (3 + k) + i] = bx[3 + k];
        }
        const int32_t cnt = b.count[2 * pn + c];
        slots[i] = cnt > 0 ? slot_word(b.child[2 * pn + c], cnt) : (uint32_t)w.next[4 * q + i];
        metas[i] = L.R > 0 ? meta_of(pn, c) : 0u;
        if (L.R > 0) {
          float* sc = reinterpret_cast<float*>(rec + 128);
          for (int k = 0; k < 3; ++k)
            sc[4 * k + i] = (float)L.R / std::fmax(bx[3 + k] - bx[k], 1e-30f);
          if (!L.compress)
            std::memcpy(rec + L.mask_off + i * L.mstride, &b.masks[((size_t)pn * 2 + c) * L.W],
                        4 * L.W);
        }
      }
    });
  } else
  parallel_for(b.nn, resolve_threads(0), 16384, [&](int64_t n) {
    uint8_t* rec = base + L.off_nodes + (size_t)n * L.node_bytes;
    float* f = reinterpret_cast<float*>(rec);
    const float* b0 = &b.box[12 * n];
    const float* b1 = b0 + 6;
    // {lo0.xy, hi0.xy} {lo1.xy, hi1.xy} {lo0.z, hi0.z, lo1.z, hi1.z}: each
    // child's x, y bounds sit in adjacent lanes for the packed slab test
    f[0] = b0[0]; f[1] = b0[1]; f[2] = b0[3]; f[3] = b0[4];
    f[4] = b1[0]; f[5] = b1[1]; f[6] = b1[3]; f[7] = b1[4];
    f[8] = b0[2]; f[9] = b0[5]; f[10] = b1[2]; f[11] = b1[5];
    uint32_t* u = reinterpret_cast<uint32_t*>(rec + 48);
    u[0] = slot_word(b.child[2 * n], b.count[2 * n]);
    u[1] = slot_word(b.child[2 * n + 1], b.count[2 * n + 1]);
    u[2] = u[3] = 0u;
    if (L.R > 0) {
      for (int c = 0; c < 2; ++c) {
        u[2 + c] = meta_of(n, c);
        if (!L.compress)
          std::memcpy(rec + L.mask_off + c * L.mstride, &b.masks[((size_t)n * 2 + c) * L.W],
                      4 * L.W);
      }
      if (L.scales) {
        // {s0.x, s0.y, s1.x, s1.y} {s0.z, s1.z, 0, 0}
        float* sc = reinterpret_cast<float*>(rec + 64);
        float v[2][3];
        for (int c = 0; c < 2; ++c)
          for (int k = 0; k < 3; ++k) {
            const float* bx = &b.box[12 * n + 6 * c];
            v[c][k] = (float)L.R / std::fmax(bx[3 + k] - bx[k], 1e-30f);
          }
        sc[0] = v[0][0]; sc[1] = v[0][1]; sc[2] = v[1][0]; sc[3] = v[1][1];
        sc[4] = v[0][2]; sc[5] = v[1][2]; sc[6] = 0.0f; sc[7] = 0.0f;
      }
    }
  });
  parallel_for(b.ntri, resolve_threads(0), 65536, [&](int64_t k) {
    float* f = reinterpret_cast<float*>(base + L.off_tris + (size_t)k * 48);
    int32_t id = b.perm[k];
    const float* t = &b.tris[9 * (size_t)id];
    f[0] = t[0]; f[1] = t[1]; f[2] = t[2];
    std::memcpy(&f[3], &id, 4);
    f[4] = t[3] - t[0]; f[5] = t[4] - t[1]; f[6] = t[5] - t[2]; f[7] = 0.0f;
    f[8] = t[6] - t[0]; f[9] = t[7] - t[1]; f[10] = t[8] - t[2]; f[11] = 0.0f;
  });
  if (L.R > 0) {
    const int R = L.R;
    const size_t R3 = (size_t)R * R * R;
    std::vector<uint32_t> lut(R3 * R3 * L.W);
    raylut_full(R, lut.data());
    for (size_t e = 0; e < R3 * R3; ++e)
      std::memcpy(base + L.off_lut + e * L.mstride, &lut[e * L.W], 4 * L.W);
    std::vector<uint64_t> P;
    raylut_pair2d(R, P);
    std::memcpy(base + L.off_pair, P.data(), 8 * P.size());
    if (L.ray2r) {
      const std::vector<uint32_t>& t2 = raylut2r_cached(R);
      const int64_t rows = (int64_t)(t2.size() / L.W);
      parallel_for(rows, resolve_threads(0), 65536, [&](int64_t e) {
        std::memcpy(base + L.off_lut2 + (size_t)e * L.mstride, &t2[(size_t)e * L.W], 4 * L.W);
      });
    }
    if (L.compress) {
      for (int j = 0; j < b.K; ++j)
        std::memcpy(base + L.off_clut + (size_t)j * L.mstride, &b.clut[(size_t)j * L.W], 4 * L.W);
      // Sec. 3.2.2: bit (row, j) = the ray mask of row meets LUT entry j
      uint32_t* bits = reinterpret_cast<uint32_t*>(base + L.off_bits);
      const int W = L.W, K = b.K;
      parallel_for((int64_t)(R3 * R3), resolve_threads(0), 1024, [&](int64_t row) {
        const uint32_t* rm = &lut[(size_t)row * W];
        uint32_t* out = bits + (size_t)row * 8;
        for (int j = 0; j < K; ++j) {
          const uint32_t* cm = &b.clut[(size_t)j * W];
          uint32_t acc = 0;
          for (int w = 0; w < W; ++w) acc |= rm[w] & cm[w];
          if (acc) out[j >> 5] |= 1u << (j & 31);
        }
      });
    }
  }
}

}  // namespace sc
