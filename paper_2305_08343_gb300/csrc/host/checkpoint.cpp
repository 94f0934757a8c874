// checkpoint.cpp — saving and loading a built BVH (host arrays, masks,
// compression LUT), so that a large build is paid once.
//
// File: "SCBVHCK1", u32 format version, u32 byte-order mark 0x01020304,
// the scalar fields, then every array as (u64 element count, raw elements),
// then a u64 FNV-1a hash of all preceding bytes.  Written to a temporary
// file and renamed into place.  Loading checks the magic, version, byte
// order, hash, array sizes and the tree's index ranges before it returns a
// handle; any mismatch is SC_ERR_IO.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace sc;

namespace {

constexpr char kMagic[8] = {'S', 'C', 'B', 'V', 'H', 'C', 'K', '1'};
constexpr uint32_t kVersion = 3, kOrder = 0x01020304u;

struct Writer {
  std::vector<uint8_t> buf;
  void raw(const void* p, size_t n) {
    const uint8_t* b = static_cast<const uint8_t*>(p);
    buf.insert(buf.end(), b, b + n);
  }
  template <class T>
  void val(const T& v) {
    raw(&v, sizeof(T));
  }
  template <class T>
  void vec(const std::vector<T>& v) {
    val<uint64_t>(v.size());
    if (!v.empty()) raw(v.data(), v.size() * sizeof(T));
  }
};

struct Reader {
  const uint8_t* p;
  size_t n, at = 0;
  void raw(void* out, size_t k) {
    if (k > n - at) fail(SC_ERR_IO, "checkpoint truncated");
    std::memcpy(out, p + at, k);
    at += k;
  }
  template <class T>
  T val() {
    T v;
    raw(&v, sizeof(T));
    return v;
  }
  template <class T>
  void vec(std::vector<T>& v, uint64_t expect) {
    const uint64_t k = val<uint64_t>();
    if (k != expect) fail(SC_ERR_IO, "checkpoint array has %llu entries, expected %llu",
                          (unsigned long long)k, (unsigned long long)expect);
    if (k > (n - at) / sizeof(T)) fail(SC_ERR_IO, "checkpoint truncated");
    v.resize(k);
    if (k) raw(v.data(), k * sizeof(T));
  }
};

uint64_t fnv1a(const uint8_t* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

void put_opts(Writer& w, const sc_build_opts& o) {
  w.val(o.max_leaf); w.val(o.bins); w.val(o.L); w.val(o.lut_size); w.val(o.chunk_bits);
  w.val(o.eps_rel); w.val(o.threads); w.val(o.skip_bits); w.val(o.test_stride);
  w.val(o.leaf_min_tris); w.val(o.gpu_masks); w.val(o.gpu_bvh);
}

void get_opts(Reader& r, sc_build_opts& o) {
  o.max_leaf = r.val<int>(); o.bins = r.val<int>(); o.L = r.val<int>();
  o.lut_size = r.val<int>(); o.chunk_bits = r.val<int>(); o.eps_rel = r.val<double>();
  o.threads = r.val<int>(); o.skip_bits = r.val<int>(); o.test_stride = r.val<int>();
  o.leaf_min_tris = r.val<int>(); o.gpu_masks = r.val<int>(); o.gpu_bvh = r.val<int>();
}

// The tree must be one a build could have made: pre-order node numbering
// (children after parents), leaves inside the triangle array.
void validate(const Bvh& b) {
  auto slot_ok = [&](int32_t child, int32_t count, int64_t parent) {
    if (count < 0 || count > kMaxLeafTris) return false;
    if (count > 0) return child >= 0 && (int64_t)child + count <= b.ntri;
    return child > parent && child < b.nn;
  };
  if (b.ntri > 0 && !slot_ok(b.root_child, b.root_count, -1))
    fail(SC_ERR_IO, "checkpoint: bad root slot");
  for (int64_t n = 0; n < b.nn; ++n)
    for (int c = 0; c < 2; ++c)
      if (!slot_ok(b.child[2 * n + c], b.count[2 * n + c], n))
        fail(SC_ERR_IO, "checkpoint: node %lld child %d out of range", (long long)n, c);
  for (int64_t i = 0; i < b.ntri; ++i)
    if (b.perm[i] < 0 || b.perm[i] >= b.ntri) fail(SC_ERR_IO, "checkpoint: bad permutation");
  if (b.compress)
    for (uint8_t k : b.cidx)
      if (k >= b.K) fail(SC_ERR_IO, "checkpoint: LUT index out of range");
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

sc_status sc_bvh_save(const sc_bvh* h, const char* path) {
  SC_TRY
  if (!h || !path) fail(SC_ERR_ARG, "sc_bvh_save: NULL argument");
  const Bvh& b = h->b;
  Writer w;
  w.raw(kMagic, sizeof(kMagic));
  w.val(kVersion);
  w.val(kOrder);
  w.val(b.ntri); w.val(b.nn); w.val(b.root_child); w.val(b.root_count);
  w.raw(b.root_box, sizeof(b.root_box));
  w.val(b.max_depth); w.val(b.R); w.val(b.L); w.val(b.W); w.val(b.compress); w.val(b.K);
  w.val(b.bits); w.val(b.eps); w.val(b.ms_bvh); w.val(b.ms_masks); w.val(b.ms_compress);
  put_opts(w, b.opts);
  w.vec(b.tris); w.vec(b.child); w.vec(b.count); w.vec(b.box); w.vec(b.perm); w.vec(b.ndepth);
  w.vec(b.masks); w.vec(b.clut); w.vec(b.cidx);
  const uint64_t hsum = fnv1a(w.buf.data(), w.buf.size());
  w.val(hsum);
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) fail(SC_ERR_IO, "cannot open %s for writing", tmp.c_str());
  const size_t put = std::fwrite(w.buf.data(), 1, w.buf.size(), f);
  const bool ok = put == w.buf.size() && std::fflush(f) == 0;
  std::fclose(f);
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    fail(SC_ERR_IO, "cannot write %s", path);
  }
  return SC_OK;
  SC_CATCH
}

sc_status sc_bvh_load(const char* path, sc_bvh** out) {
  SC_TRY
  if (!path || !out) fail(SC_ERR_ARG, "sc_bvh_load: NULL argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) fail(SC_ERR_IO, "cannot open %s", path);
  std::vector<uint8_t> data;
  uint8_t chunk[1 << 16];
  size_t got;
  while ((got = std::fread(chunk, 1, sizeof(chunk), f)) > 0) data.insert(data.end(), chunk, chunk + got);
  const bool err = std::ferror(f) != 0;
  std::fclose(f);
  if (err) fail(SC_ERR_IO, "cannot read %s", path);
  if (data.size() < sizeof(kMagic) + 16) fail(SC_ERR_IO, "%s: not a BVH checkpoint", path);
  uint64_t stored;
  std::memcpy(&stored, data.data() + data.size() - 8, 8);
  if (fnv1a(data.data(), data.size() - 8) != stored) fail(SC_ERR_IO, "%s: checksum mismatch", path);
  Reader r{data.data(), data.size() - 8};
  char magic[8];
  r.raw(magic, 8);
  if (std::memcmp(magic, kMagic, 8) != 0) fail(SC_ERR_IO, "%s: not a BVH checkpoint", path);
  if (r.val<uint32_t>() != kVersion) fail(SC_ERR_IO, "%s: unsupported checkpoint version", path);
  if (r.val<uint32_t>() != kOrder) fail(SC_ERR_IO, "%s: written with another byte order", path);
  sc_bvh* h = new sc_bvh();
  try {
    Bvh& b = h->b;
    b.ntri = r.val<int64_t>(); b.nn = r.val<int64_t>();
    b.root_child = r.val<int32_t>(); b.root_count = r.val<int32_t>();
    r.raw(b.root_box, sizeof(b.root_box));
    b.max_depth = r.val<int>(); b.R = r.val<int>(); b.L = r.val<int>(); b.W = r.val<int>();
    b.compress = r.val<int>(); b.K = r.val<int>(); b.bits = r.val<int>();
    b.eps = r.val<double>(); b.ms_bvh = r.val<double>(); b.ms_masks = r.val<double>();
    b.ms_compress = r.val<double>();
    get_opts(r, b.opts);
    if (b.ntri < 0 || b.ntri >= kMaxTris || b.nn < 0 || b.nn > 2 * b.ntri + 1 ||
        !(b.R == 0 || b.R == 4 || b.R == 6 || b.R == 8) || b.W != (b.R ? mask_words(b.R) : 0) ||
        b.K < 0 || b.K > 256 || (b.compress && (b.R == 0 || b.K < 1)))
      fail(SC_ERR_IO, "%s: inconsistent header", path);
    const uint64_t nn = (uint64_t)b.nn, W = (uint64_t)b.W;
    r.vec(b.tris, 9 * (uint64_t)b.ntri);
    r.vec(b.child, 2 * nn);
    r.vec(b.count, 2 * nn);
    r.vec(b.box, 12 * nn);
    r.vec(b.perm, (uint64_t)b.ntri);
    r.vec(b.ndepth, nn);
    r.vec(b.masks, b.R ? 2 * nn * W : 0);
    r.vec(b.clut, b.compress ? (uint64_t)b.K * W : 0);
    r.vec(b.cidx, b.compress ? 2 * nn : 0);
    if (r.at != r.n) fail(SC_ERR_IO, "%s: trailing bytes", path);
    validate(b);
  } catch (...) {
    delete h;
    throw;
  }
  *out = h;
  return SC_OK;
  SC_CATCH
}

}  // extern "C"
