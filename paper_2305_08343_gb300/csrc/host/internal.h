// internal.h — host-side data structures and helpers of libsubcull.
#pragma once

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "subcull.h"

namespace sc {

// ---------------------------------------------------------------- errors --
void set_error(const char* fmt, ...);
void clear_error();

// Thrown inside the library only; converted to sc_status at the boundary.
struct Error {
  sc_status code;
  std::string msg;
};
[[noreturn]] void fail(sc_status code, const char* fmt, ...);

// --------------------------------------------------------------- threads --
int resolve_threads(int requested);
// Runs fn(i) for i in [0, n) on `threads` threads, indices handed out in
// blocks of `grain` by an atomic counter.
void parallel_for(int64_t n, int threads, int64_t grain,
                  const std::function<void(int64_t)>& fn);
// Runs fn(begin, end, part) over `parts` contiguous ranges of [0, n).
void parallel_ranges(int64_t n, int parts,
                     const std::function<void(int64_t, int64_t, int)>& fn);

double now_ms();

// ----------------------------------------------------------------- masks --
inline int mask_words(int R) { return (R * R * R + 31) / 32; }
// Bytes of one mask in the device image: R=4 -> 8, R=6 -> 32, R=8 -> 64.
inline int mask_stride(int R) {
  int b = mask_words(R) * 4;
  return b <= 8 ? 8 : (b <= 32 ? 32 : 64);
}

// ------------------------------------------------------------------- BVH --
struct Bvh {
  int64_t ntri = 0;
  std::vector<float> tris;  // input order, [ntri][9]
  int32_t root_child = -1, root_count = 0;
  float root_box[6] = {0, 0, 0, 0, 0, 0};
  int64_t nn = 0;               // inner nodes (child-pair records)
  std::vector<int32_t> child;   // [nn][2]
  std::vector<int32_t> count;   // [nn][2]
  std::vector<float> box;       // [nn][2][6]
  std::vector<int32_t> perm;    // [ntri] triangle id at each leaf position
  std::vector<int32_t> ndepth;  // [nn] depth of the slot the node fills
  int max_depth = 0;
  // object masks
  int R = 0, L = 3, W = 0;
  double eps = 0.0;
  std::vector<uint32_t> masks;  // [nn][2][W]
  // compression
  int compress = 0, K = 0, bits = 8;
  std::vector<uint32_t> clut;   // [K][W]
  std::vector<uint8_t> cidx;    // [nn][2]
  double ms_bvh = 0, ms_masks = 0, ms_compress = 0;
  sc_build_opts opts{};
};

void build_bvh(Bvh& b, const float* tris, int64_t n, int max_leaf, int bins,
               int threads);
// The same tree built on the current GPU (bins <= 32).
void build_bvh_gpu(Bvh& b, const float* tris, int64_t n, int max_leaf, int bins);
void build_masks(Bvh& b, int R, int L, double eps, int threads);
// The same masks built on the current GPU (bit-identical).
void build_masks_gpu(Bvh& b, int R, int L, double eps);
void build_compression(Bvh& b, int K, int bits, int threads);
// Refit support: masks of the marked nodes only (host or GPU), and Alg. 3
// against the existing LUT for the marked nodes' slots (all when NULL).
void refit_masks(Bvh& b, const std::vector<uint8_t>& node_dirty, int threads);
void refit_masks_gpu(Bvh& b, const std::vector<uint8_t>& node_dirty);
void encode_slots(Bvh& b, int threads, const std::vector<uint8_t>* node_dirty);
double scene_eps(const float* tris, int64_t n, double eps_rel);

// Ray-mask tables (Sec. 3.1.1).  pair2d: [R^4] entries of R^2 bits,
// index ((ba*R + bb)*R + ea)*R + eb, bit va + R*vb.  full: [R^6][W].
void raylut_pair2d(int R, std::vector<uint64_t>& out);
void raylut_full(int R, uint32_t* out);
// The R_ray = 2R table (Sec. 4.2): [(2R)^6][W], row beg*(2R)^3 + end over
// cells of the 2R grid, each row an R^3-bit mask.
void raylut2r_full(int R, uint32_t* out);

// ---------------------------------------------------------- device image --
// Node record (child pair), 16-byte aligned, fetched as float4s:
//   f0 = {lo0.x, lo0.y, hi0.x, hi0.y}  f1 = {lo1.x, lo1.y, hi1.x, hi1.y}
//   f2 = {lo0.z, hi0.z, lo1.z, hi1.z}  f3 = {slot0, slot1, meta0, meta1}
// slot: inner -> child node index (>= 0); leaf -> 0x80000000 |
// (count-1) << 28 | first triangle position.  meta: compression LUT index.
// meta bit 8: the child's (decoded) mask is all ones, so its culling test
// cannot remove it.  SC_LAYOUT_MASKED stores the scales R / max(extent,
// 1e-30) of both children at +64 as {s0.x, s0.y, s1.x, s1.y} {s0.z, s1.z,
// 0, 0}; the two uncompressed
// masks follow at mask_off and mask_off + mask_stride.
constexpr uint32_t kLeafBit = 0x80000000u;
constexpr uint32_t kMetaFull = 0x100u;
constexpr int kMaxLeafTris = 8;
constexpr int64_t kMaxTris = int64_t(1) << 28;

struct ImageLayout {
  int layout = 0;          // SC_LAYOUT_*
  int width = 2;           // children per node record (2, or 4 for the *4 layouts)
  int64_t nodes = 0;       // node records in the image
  int stack_need = 0;      // deepest possible traversal stack
  int R = 0, W = 0, mstride = 0, compress = 0, K = 0;
  int scales = 0;          // per-child Alg. 1 scales stored at +64
  int ray2r = 0;           // the image also holds the R_ray = 2R table
  int mask_off = 64;       // first object mask inside a node record
  int node_bytes = 64;
  size_t off_nodes = 0, off_tris = 0, off_lut = 0, off_pair = 0, off_clut = 0, off_bits = 0;
  size_t off_lut2 = 0;
  size_t total = 0;
};
ImageLayout image_layout(const Bvh& b, int layout);
void pack_image(const Bvh& b, const ImageLayout& L, std::vector<uint8_t>& img);
uint32_t root_slot_word(const Bvh& b);

}  // namespace sc

// Host view of an uploaded image (defined for the C-ABI's opaque type).
struct sc_dbvh {
  const uint8_t* base = nullptr;
  sc::ImageLayout lay;
  int64_t ntri = 0, nn = 0;
  uint32_t root_slot = 0;
  int has_root = 0;
  int stack_need = 0;  // max_depth + 1
  float root_box[6] = {0, 0, 0, 0, 0, 0};  // scene box (lo.xyz, hi.xyz)
};

struct sc_bvh {
  sc::Bvh b;
};
