// trace_api.cu — device entry points of the C-ABI: image upload, trace
// launches, the end-to-end host-buffer form and the status poll.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "host/internal.h"
#include "trace_kernel.cuh"

namespace sct {
KernelFn get_kernel_plain(int mode);
KernelFn get_kernel_r4(int cull, int mode, int lutv, int scales);
KernelFn get_kernel_r6(int cull, int mode, int lutv, int scales);
KernelFn get_kernel_r8(int cull, int mode, int lutv, int scales);
WaveKernelFn get_waves_plain(int block, int stack);
WaveKernelFn get_waves_r4(int cull, int lutv, int scales);
WaveKernelFn get_waves_r6(int cull, int lutv, int scales, int block, int stack);
WaveKernelFn get_waves_r8(int cull, int lutv, int scales);
SeededKernelFn get_seeded_plain();
KernelFn get_kernel_w4_plain(int mode);
KernelFn get_kernel_w4_r4(int cull, int mode, int lutv);
KernelFn get_kernel_w4_r6(int cull, int mode, int lutv);
KernelFn get_kernel_w4_r8(int cull, int mode, int lutv);
WaveKernelFn get_waves_w4_plain(int block);
WaveKernelFn get_waves_w4_r4(int cull, int lutv, int block);
WaveKernelFn get_waves_w4_r6(int cull, int lutv, int block);
WaveKernelFn get_waves_w4_r8(int cull, int lutv, int block);
SeededKernelFn get_seeded_r4(int cull, int lutv, int scales);
SeededKernelFn get_seeded_r6(int cull, int lutv, int scales);
SeededKernelFn get_seeded_r8(int cull, int lutv, int scales);
bool var_supported(int opt);
KernelFn get_kernel_var(int R, int cull, int mode, int lutv, int opt);
WaveKernelFn get_waves_var(int R, int cull, int lutv, int opt);
}  // namespace sct

using namespace sc;

namespace {

constexpr int kBlock = sct::kBlock;
constexpr size_t kWorkBytes = 256;
constexpr int kDefaultRefill = 8;

#define CUDA_OK(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      fail(SC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

struct DevInfo {
  int sms = 0;
};

DevInfo device_info() {
  int dev = 0;
  CUDA_OK(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::vector<DevInfo> cache;
  std::lock_guard<std::mutex> g(mu);
  if ((int)cache.size() <= dev) cache.resize(dev + 1);
  if (cache[dev].sms == 0) {
    int sms = 0;
    CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cache[dev].sms = sms;
  }
  return cache[dev];
}

// Ray-mask lookup variant: 0 full table (global), 1 shared memory (the full
// table at R = 4, the factored tables otherwise), 2 bit table (compressed
// images only), 4 the R_ray = 2R table (images that hold it), 5 the
// factored tables read through L1 (binary R = 6 uncompressed images with
// stored scales).  AUTO: the 2R
// table when present, else the bit table when compressed, else the full
// table (shared-memory tables take the L1 capacity the node fetches need).
int lut_variant(const sc_dbvh* d, int lut_mode) {
  switch (lut_mode) {
    case SC_LUT_AUTO: return d->lay.ray2r ? 4 : (d->lay.compress ? 2 : 0);
    case SC_LUT_GLOBAL: return 0;
    case SC_LUT_SHARED: return 1;
    case SC_LUT_BITTABLE:
      if (!d->lay.compress) fail(SC_ERR_ARG, "the bit table needs a compressed image");
      return 2;
    case SC_LUT_RAY2R:
      if (!d->lay.ray2r) fail(SC_ERR_ARG, "the R_ray = 2R table needs an SC_LAYOUT_MASKED_RAY2R image");
      return 4;
    case SC_LUT_FACTORED_L1:
      if (d->lay.R != 6 || d->lay.compress || !d->lay.scales || d->lay.width != 2)
        fail(SC_ERR_UNSUPPORTED,
             "the L1-read factored tables are built for binary R = 6 images with uncompressed "
             "masks and stored scales");
      return 5;
  }
  fail(SC_ERR_ARG, "bad lut_mode %d", lut_mode);
}

sct::KernelFn pick_kernel(const sc_dbvh* d, int mode, int cull, int lutv) {
  if (d->lay.width == 4) {
    if (!cull) return sct::get_kernel_w4_plain(mode);
    const int c = d->lay.compress ? 2 : 1;
    const int lv = lutv == 2 ? 2 : 0;  // 4-wide: global table or bit table
    switch (d->lay.R) {
      case 4: return sct::get_kernel_w4_r4(c, mode, lv);
      case 6: return sct::get_kernel_w4_r6(c, mode, lv);
      case 8: return sct::get_kernel_w4_r8(c, mode, lv);
    }
    fail(SC_ERR_UNSUPPORTED, "no 4-wide kernel for R = %d", d->lay.R);
  }
  if (!cull) return sct::get_kernel_plain(mode);
  int c = d->lay.compress ? 2 : 1;
  const int sc = d->lay.scales;
  switch (d->lay.R) {
    case 4: return sct::get_kernel_r4(c, mode, lutv, sc);
    case 6: return sct::get_kernel_r6(c, mode, lutv, sc);
    case 8: return sct::get_kernel_r8(c, mode, lutv, sc);
  }
  fail(SC_ERR_UNSUPPORTED, "no kernel for R = %d", d->lay.R);
}

// Kernels with non-default options (sc_trace_opts.variant): R = 6 images
// with the full table (uncompressed) or the bit table (compressed), scales
// stored, and the plain traversal.
bool variant_image_ok(const sc_dbvh* d, int cull, int lutv) {
  if (d->lay.width != 2) return false;
  return !cull || (d->lay.R == 6 && d->lay.scales &&
                   ((!d->lay.compress && lutv == 0) || (d->lay.compress && lutv == 2)));
}

void check_variant(const sc_dbvh* d, int cull, int lutv, int variant) {
  if (!sct::var_supported(variant))
    fail(SC_ERR_UNSUPPORTED, "kernel variant %d is not built", variant);
  if (d->lay.width != 2) fail(SC_ERR_UNSUPPORTED, "kernel variants need a binary image");
  if (!variant_image_ok(d, cull, lutv))
    fail(SC_ERR_UNSUPPORTED,
         "kernel variants are built for R = 6 images with stored scales (full table "
         "uncompressed, bit table compressed)");
}

sct::KernelFn pick_kernel_var(const sc_dbvh* d, int mode, int cull, int lutv, int variant) {
  check_variant(d, cull, lutv, variant);
  sct::KernelFn k = cull ? sct::get_kernel_var(6, d->lay.compress ? 2 : 1, mode, lutv, variant)
                         : sct::get_kernel_var(0, 0, mode, 0, variant);
  if (!k) fail(SC_ERR_UNSUPPORTED, "kernel variant %d is not built for this image", variant);
  return k;
}

void launch_trace(const sc_dbvh* d, const float* d_rays, int64_t n, sc_hit* d_hits,
                  uint32_t* d_counts, int mode, int cull, const sc_trace_opts* opts,
                  void* d_work, size_t work_bytes, cudaStream_t st) {
  if (!d) fail(SC_ERR_ARG, "sc_trace: NULL device BVH");
  if (n < 0 || n > (int64_t)0x7FFFFF00) fail(SC_ERR_ARG, "sc_trace: n out of range");
  if (n > 0 && (!d_rays || !d_hits)) fail(SC_ERR_ARG, "sc_trace: NULL rays or hits");
  if (!d_work || work_bytes < kWorkBytes) fail(SC_ERR_ARG, "sc_trace: workspace too small");
  if ((reinterpret_cast<uintptr_t>(d_rays) & 15) || (reinterpret_cast<uintptr_t>(d_hits) & 15) ||
      (reinterpret_cast<uintptr_t>(d_counts) & 7) || (reinterpret_cast<uintptr_t>(d_work) & 15))
    fail(SC_ERR_ARG, "sc_trace: rays/hits/workspace must be 16-byte aligned, counts 8-byte");
  if (mode != SC_CLOSEST && mode != SC_ANY) fail(SC_ERR_ARG, "sc_trace: bad mode %d", mode);
  if (cull && d->lay.R == 0)
    fail(SC_ERR_STATE, "sc_trace: culling needs an image uploaded with a masked layout");
  if (d->stack_need > sct::kStack)
    fail(SC_ERR_UNSUPPORTED, "BVH depth %d exceeds the traversal stack (%d)", d->stack_need,
         sct::kStack);
  sc_trace_opts o{};
  o.lut_mode = SC_LUT_AUTO;
  if (opts) o = *opts;
  if (o.block != 0 && o.block != kBlock) fail(SC_ERR_UNSUPPORTED, "block must be 0 or 128");
  if (o.stack != 0 && o.stack != sct::kStack) fail(SC_ERR_UNSUPPORTED, "stack must be 0 or 64");
  if (o.refill < 0 || o.refill > 32) fail(SC_ERR_ARG, "refill must be 0..32");
  const int lutv = lut_variant(d, o.lut_mode);
  sct::KernelFn k = o.variant ? pick_kernel_var(d, mode, cull ? 1 : 0, lutv, o.variant)
                              : pick_kernel(d, mode, cull ? 1 : 0, lutv);
  CUDA_OK(cudaMemsetAsync(d_work, 0, kWorkBytes, st));
  if (n == 0) return;
  DevInfo di = device_info();
  int per_sm = o.blocks_per_sm;
  if (per_sm <= 0) {
    CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k, kBlock, 0));
    if (per_sm < 1) per_sm = 1;
  }
  int64_t need = (n + kBlock - 1) / kBlock;
  int64_t grid = (int64_t)di.sms * per_sm;
  if (grid > need) grid = need;
  sct::Params p;
  const uint8_t* base = d->base;
  p.nodes = reinterpret_cast<const float4*>(base + d->lay.off_nodes);
  p.node_f4 = d->lay.node_bytes / 16;
  p.mask_off_f4 = d->lay.mask_off / 16;
  p.tris = reinterpret_cast<const float4*>(base + d->lay.off_tris);
  p.lut = d->lay.R ? reinterpret_cast<const uint4*>(base + d->lay.off_lut) : nullptr;
  p.pair = d->lay.R ? reinterpret_cast<const uint2*>(base + d->lay.off_pair) : nullptr;
  p.clut = d->lay.compress ? reinterpret_cast<const uint4*>(base + d->lay.off_clut) : nullptr;
  p.bits = d->lay.compress ? reinterpret_cast<const uint32_t*>(base + d->lay.off_bits) : nullptr;
  p.lut2 = d->lay.ray2r ? reinterpret_cast<const uint4*>(base + d->lay.off_lut2) : nullptr;
  p.rays = reinterpret_cast<const float4*>(d_rays);
  p.hits = reinterpret_cast<float4*>(d_hits);
  p.counts = reinterpret_cast<uint2*>(d_counts);
  p.work = reinterpret_cast<unsigned*>(d_work);
  p.status = p.work + 1;
  p.n = n;
  p.num_nodes = d->nn;
  p.num_tris = d->ntri;
  p.root_slot = d->root_slot;
  p.has_root = d->has_root;
  p.refill = o.refill ? o.refill : kDefaultRefill;
  k<<<(unsigned)grid, kBlock, 0, st>>>(p);
  CUDA_OK(cudaGetLastError());
}

int64_t wave_chunk_of(int64_t n0, const sc_trace_opts* o) {
  int64_t c = (o && o->wave_chunk > 0) ? o->wave_chunk : n0;
  if (c > n0) c = n0;
  return c > 0 ? c : 1;
}

size_t waves_ctrl_bytes(int64_t n0, int64_t chunk) {
  const int64_t nch = n0 > 0 ? (n0 + chunk - 1) / chunk : 1;
  return ((size_t)(sct::WW_HEAD + sct::WW_CHUNK_WORDS * nch) * 4 + 255) / 256 * 256;
}

size_t waves_ws_bytes(int64_t n0, int64_t chunk) {
  const size_t q = (size_t)(chunk > 0 ? chunk : 1);
  return waves_ctrl_bytes(n0, chunk) + 3 * ((q * 32 + 255) / 256 * 256) +
         3 * ((q * 4 + 255) / 256 * 256) + (size_t)sct::kSortBins * 4;
}

void fill_params(const sc_dbvh* d, sct::Params& p) {
  const uint8_t* base = d->base;
  p.nodes = reinterpret_cast<const float4*>(base + d->lay.off_nodes);
  p.node_f4 = d->lay.node_bytes / 16;
  p.mask_off_f4 = d->lay.mask_off / 16;
  p.tris = reinterpret_cast<const float4*>(base + d->lay.off_tris);
  p.lut = d->lay.R ? reinterpret_cast<const uint4*>(base + d->lay.off_lut) : nullptr;
  p.pair = d->lay.R ? reinterpret_cast<const uint2*>(base + d->lay.off_pair) : nullptr;
  p.clut = d->lay.compress ? reinterpret_cast<const uint4*>(base + d->lay.off_clut) : nullptr;
  p.bits = d->lay.compress ? reinterpret_cast<const uint32_t*>(base + d->lay.off_bits) : nullptr;
  p.lut2 = d->lay.ray2r ? reinterpret_cast<const uint4*>(base + d->lay.off_lut2) : nullptr;
  p.num_nodes = d->nn;
  p.num_tris = d->ntri;
  p.root_slot = d->root_slot;
  p.has_root = d->has_root;
}

// The lookup variant of a wave launch: the factored tables in shared memory
// are built for the wave pipeline only at R = 6 with uncompressed masks and
// stored scales (and at R = 4 as the full table); the full table elsewhere.
int waves_lutv(const sc_dbvh* d, int lut_mode) {
  int lutv = lut_variant(d, lut_mode);
  if (lutv == 1 && d->lay.R != 4 && !(d->lay.R == 6 && !d->lay.compress && d->lay.scales))
    lutv = 0;
  return lutv;
}

sct::WaveKernelFn pick_waves(const sc_dbvh* d, int cull, int lutv, int block, int stack) {
  if (d->lay.width == 4) {
    if (block == 64 || stack != 64)
      fail(SC_ERR_UNSUPPORTED, "4-wide wave kernels: blocks of 128 / 256, stack 64");
    if (!cull) return sct::get_waves_w4_plain(block);
    const int c = d->lay.compress ? 2 : 1;
    const int lv = lutv == 2 ? 2 : 0;
    switch (d->lay.R) {
      case 4: return sct::get_waves_w4_r4(c, lv, block);
      case 6: return sct::get_waves_w4_r6(c, lv, block);
      case 8: return sct::get_waves_w4_r8(c, lv, block);
    }
    fail(SC_ERR_UNSUPPORTED, "no 4-wide wave kernel for R = %d", d->lay.R);
  }
  const bool tuned = block != kBlock || stack != sct::kStack;
  if (!cull) return sct::get_waves_plain(block, stack);
  const int c = d->lay.compress ? 2 : 1, sc = d->lay.scales;
  if (d->lay.R == 6) return sct::get_waves_r6(c, lutv, sc, block, stack);
  if (tuned)
    fail(SC_ERR_UNSUPPORTED, "block %d / stack %d wave kernels exist for R = 6 and plain only",
         block, stack);
  switch (d->lay.R) {
    case 4: return sct::get_waves_r4(c, lutv, sc);
    case 8: return sct::get_waves_r8(c, lutv, sc);
  }
  fail(SC_ERR_UNSUPPORTED, "no wave kernel for R = %d", d->lay.R);
}

void launch_waves(const sc_dbvh* d, const float* d_rays, int64_t n0, int bounces, uint32_t seed,
                  int cull, const sc_wave_out* outs, const sc_trace_opts* opts, void* d_ws,
                  size_t ws_bytes, cudaStream_t st) {
  if (!d) fail(SC_ERR_ARG, "sc_trace_waves: NULL device BVH");
  if (n0 < 0 || n0 > (int64_t)0x7FFFFF00) fail(SC_ERR_ARG, "sc_trace_waves: n0 out of range");
  if (bounces < 0 || bounces + 1 > sct::kMaxWaves)
    fail(SC_ERR_ARG, "sc_trace_waves: bounces must be 0..%d", sct::kMaxWaves - 1);
  if (!outs) fail(SC_ERR_ARG, "sc_trace_waves: NULL outputs");
  for (int w = 0; w <= bounces; ++w) {
    if (n0 > 0 && !outs[w].hits) fail(SC_ERR_ARG, "sc_trace_waves: wave %d has no hit buffer", w);
    if ((reinterpret_cast<uintptr_t>(outs[w].hits) & 15) ||
        (reinterpret_cast<uintptr_t>(outs[w].counts) & 7) ||
        (reinterpret_cast<uintptr_t>(outs[w].path) & 3))
      fail(SC_ERR_ARG, "sc_trace_waves: misaligned output of wave %d", w);
  }
  if (n0 > 0 && !d_rays) fail(SC_ERR_ARG, "sc_trace_waves: NULL rays");
  if (reinterpret_cast<uintptr_t>(d_rays) & 15) fail(SC_ERR_ARG, "rays must be 16-byte aligned");
  sc_trace_opts o{};
  o.lut_mode = SC_LUT_AUTO;
  if (opts) o = *opts;
  const int64_t chunk = wave_chunk_of(n0, &o);
  if (o.wave_chunk < 0) fail(SC_ERR_ARG, "wave_chunk must be >= 0");
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255) || ws_bytes < waves_ws_bytes(n0, chunk))
    fail(SC_ERR_ARG, "sc_trace_waves: workspace must be 256-byte aligned and >= %zu bytes",
         waves_ws_bytes(n0, chunk));
  if (cull && d->lay.R == 0) fail(SC_ERR_STATE, "sc_trace_waves: culling needs a masked image");
  const int block = o.block ? o.block : kBlock;
  const int stack = o.stack ? o.stack : sct::kStack;
  if (block != 64 && block != 128 && block != 256) fail(SC_ERR_ARG, "block must be 64, 128 or 256");
  if (stack != 32 && stack != 64) fail(SC_ERR_ARG, "stack must be 32 or 64");
  if (d->stack_need > stack)
    fail(SC_ERR_UNSUPPORTED, "BVH depth %d exceeds the traversal stack (%d)", d->stack_need,
         stack);
  if (o.refill < 0 || o.refill > 32) fail(SC_ERR_ARG, "refill must be 0..32");
  const int lutv = waves_lutv(d, o.lut_mode);
  sct::WaveKernelFn k = nullptr;
  if (o.variant) {
    check_variant(d, cull, lutv, o.variant);
    if (block != kBlock || stack != sct::kStack)
      fail(SC_ERR_UNSUPPORTED, "kernel variants of the waves are built for block %d, stack %d",
           kBlock, sct::kStack);
    k = cull ? sct::get_waves_var(6, d->lay.compress ? 2 : 1, lutv, o.variant)
             : sct::get_waves_var(0, 0, 0, o.variant);
  } else {
    k = pick_waves(d, cull, lutv, block, stack);
  }
  if (!k) fail(SC_ERR_UNSUPPORTED, "no wave kernel for this block / stack / lookup combination");
  const size_t ctrl = waves_ctrl_bytes(n0, chunk);
  CUDA_OK(cudaMemsetAsync(d_ws, 0, ctrl, st));
  if (n0 == 0) return;
  sct::WaveParams wp;
  std::memset(&wp, 0, sizeof(wp));
  fill_params(d, wp.p);
  wp.p.work = reinterpret_cast<unsigned*>(d_ws);
  wp.p.status = wp.p.work + sct::WW_STATUS;
  wp.p.refill = o.refill ? o.refill : kDefaultRefill;
  wp.p.n = n0;
  uint8_t* ws = reinterpret_cast<uint8_t*>(d_ws);
  const size_t q = (size_t)chunk;
  size_t off = ctrl;
  for (int i = 0; i < 2; ++i) {
    wp.qrays[i] = reinterpret_cast<float4*>(ws + off);
    off += (q * 32 + 255) / 256 * 256;
  }
  for (int i = 0; i < 2; ++i) {
    wp.qpath[i] = reinterpret_cast<int*>(ws + off);
    off += (q * 4 + 255) / 256 * 256;
  }
  wp.srays = reinterpret_cast<float4*>(ws + off);
  off += (q * 32 + 255) / 256 * 256;
  wp.spath = reinterpret_cast<int*>(ws + off);
  off += (q * 4 + 255) / 256 * 256;
  wp.hist = reinterpret_cast<unsigned*>(ws + off);
  for (int k = 0; k < 3; ++k) {
    const float ext = d->root_box[3 + k] - d->root_box[k];
    wp.box_lo[k] = d->root_box[k];
    wp.box_scale[k] = ext > 0.0f ? (float)(1 << sct::kSortCellBits) / ext : 0.0f;
  }
  wp.rays0 = reinterpret_cast<const float4*>(d_rays);
  wp.n0 = n0;
  wp.chunk = chunk;
  for (int w = 0; w <= bounces; ++w) {
    wp.hits[w] = reinterpret_cast<float4*>(outs[w].hits);
    wp.path[w] = outs[w].path;
    wp.counts[w] = reinterpret_cast<uint2*>(outs[w].counts);
    wp.orays[w] = reinterpret_cast<float4*>(outs[w].rays);
    if (reinterpret_cast<uintptr_t>(outs[w].rays) & 15)
      fail(SC_ERR_ARG, "sc_trace_waves: misaligned ray output of wave %d", w);
  }
  wp.bounces = bounces;
  wp.seed = seed;
  wp.timeout_ns = o.wait_timeout_ns > 0 ? (unsigned long long)o.wait_timeout_ns : 2000000000ULL;
  DevInfo di = device_info();
  int per_sm = 0;
  CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k, block, 0));
  if (per_sm < 1) fail(SC_ERR_CUDA, "wave kernel cannot be resident");
  if (o.blocks_per_sm > 0 && o.blocks_per_sm < per_sm) per_sm = o.blocks_per_sm;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)(di.sms * per_sm));
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CUDA_OK(cudaLaunchKernelEx(&cfg, k, wp));
}

}  // namespace

// ---------------------------------------------------------------------------
// Scratch for sc_trace_noalloc: the ray counter and device status word that
// sc_trace keeps in a caller-provided workspace live here instead.  Every GPU
// that loads this library holds these bytes until the process exits.  Host
// code must not pass `g_noalloc_scratch` itself to a kernel (on the host it
// names a stand-in, not device memory); its device address is looked up once
// per device with cudaGetSymbolAddress, with that device current.
namespace {

constexpr size_t kNoallocScratchBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

void* noalloc_scratch_address() {
  int dev = 0;
  CUDA_OK(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::vector<void*> addr;
  std::lock_guard<std::mutex> g(mu);
  if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
  if (!addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      fail(SC_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
    addr[dev] = p;
  }
  return addr[dev];
}

}  // namespace

#define SC_TRY \
  try {        \
    clear_error();
#define SC_CATCH                              \
  }                                           \
  catch (const Error& e) {                    \
    set_error("%s", e.msg.c_str());           \
    return e.code;                            \
  }                                           \
  catch (const std::bad_alloc&) {             \
    set_error("host allocation failed");      \
    return SC_ERR_NOMEM;                      \
  }                                           \
  catch (...) {                               \
    set_error("unexpected internal error");   \
    return SC_ERR_STATE;                      \
  }

extern "C" {

sc_status sc_bvh_upload(const sc_bvh* h, int layout, void* d_buf, size_t nbytes, void* stream,
                        sc_dbvh** out) {
  SC_TRY
  if (!h || !d_buf || !out) fail(SC_ERR_ARG, "sc_bvh_upload: NULL argument");
  *out = nullptr;
  if (reinterpret_cast<uintptr_t>(d_buf) & 255) fail(SC_ERR_ARG, "d_buf must be 256-byte aligned");
  const Bvh& b = h->b;
  ImageLayout L = image_layout(b, layout);
  if (nbytes < L.total) fail(SC_ERR_NOMEM, "image needs %zu bytes, buffer has %zu", L.total, nbytes);
  std::vector<uint8_t> img;
  pack_image(b, L, img);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CUDA_OK(cudaMemcpyAsync(d_buf, img.data(), img.size(), cudaMemcpyHostToDevice, st));
  CUDA_OK(cudaStreamSynchronize(st));
  sc_dbvh* d = new sc_dbvh();
  d->base = reinterpret_cast<const uint8_t*>(d_buf);
  d->lay = L;
  d->ntri = b.ntri;
  d->nn = L.nodes;
  d->root_slot = root_slot_word(b);  // the root node is record 0 at either width
  d->has_root = b.ntri > 0 ? 1 : 0;
  d->stack_need = L.stack_need;
  for (int k = 0; k < 6; ++k) d->root_box[k] = b.root_box[k];
  *out = d;
  return SC_OK;
  SC_CATCH
}

void sc_dbvh_destroy(sc_dbvh* d) { delete d; }

size_t sc_trace_workspace_bytes(void) { return kWorkBytes; }

sc_status sc_trace(const sc_dbvh* d, const float* d_rays, int64_t n, sc_hit* d_hits,
                   uint32_t* d_counts, int mode, int cull, const sc_trace_opts* opts, void* d_work,
                   size_t work_bytes, void* stream) {
  SC_TRY
  launch_trace(d, d_rays, n, d_hits, d_counts, mode, cull, opts, d_work, work_bytes,
               reinterpret_cast<cudaStream_t>(stream));
  return SC_OK;
  SC_CATCH
}

sc_status sc_trace_seeded(const sc_dbvh* d, const float* d_rays, int64_t n, const int32_t* d_cls,
                          const sc_frontier_entry* d_frontier, int n_frontier, sc_hit* d_hits,
                          uint32_t* d_counts, int cull, const sc_trace_opts* opts, void* d_work,
                          size_t work_bytes, void* stream) {
  SC_TRY
  if (!d) fail(SC_ERR_ARG, "sc_trace_seeded: NULL device BVH");
  if (n < 0 || n > (int64_t)0x7FFFFF00) fail(SC_ERR_ARG, "sc_trace_seeded: n out of range");
  if (n > 0 && (!d_rays || !d_hits || !d_cls || !d_frontier))
    fail(SC_ERR_ARG, "sc_trace_seeded: NULL buffer");
  if (n_frontier < 1 || n_frontier > 256) fail(SC_ERR_ARG, "sc_trace_seeded: n_frontier 1..256");
  if (!d_work || work_bytes < kWorkBytes) fail(SC_ERR_ARG, "sc_trace_seeded: workspace too small");
  if ((reinterpret_cast<uintptr_t>(d_rays) & 15) || (reinterpret_cast<uintptr_t>(d_hits) & 15) ||
      (reinterpret_cast<uintptr_t>(d_counts) & 7) || (reinterpret_cast<uintptr_t>(d_frontier) & 15))
    fail(SC_ERR_ARG, "sc_trace_seeded: misaligned buffer");
  if (cull && d->lay.R == 0) fail(SC_ERR_STATE, "sc_trace_seeded: culling needs a masked image");
  if (d->lay.width != 2)
    fail(SC_ERR_UNSUPPORTED, "sc_trace_seeded: the frontier refers to binary nodes (2-wide image)");
  if (d->stack_need > sct::kStack)
    fail(SC_ERR_UNSUPPORTED, "BVH depth %d exceeds the traversal stack (%d)", d->stack_need,
         sct::kStack);
  sc_trace_opts o{};
  o.lut_mode = SC_LUT_AUTO;
  if (opts) o = *opts;
  if ((o.block && o.block != kBlock) || (o.stack && o.stack != sct::kStack))
    fail(SC_ERR_UNSUPPORTED, "sc_trace_seeded: default block and stack only");
  if (o.variant) fail(SC_ERR_UNSUPPORTED, "sc_trace_seeded: kernel variants are not built");
  if (o.refill < 0 || o.refill > 32) fail(SC_ERR_ARG, "refill must be 0..32");
  int lutv = lut_variant(d, o.lut_mode);
  if (lutv == 1 || lutv == 3 || lutv == 5) lutv = 0;  // seeded traces: the full table
  sct::SeededKernelFn k = nullptr;
  if (!cull) {
    k = sct::get_seeded_plain();
  } else {
    const int c = d->lay.compress ? 2 : 1, sc = d->lay.scales;
    switch (d->lay.R) {
      case 4: k = sct::get_seeded_r4(c, lutv, sc); break;
      case 6: k = sct::get_seeded_r6(c, lutv, sc); break;
      case 8: k = sct::get_seeded_r8(c, lutv, sc); break;
      default: fail(SC_ERR_UNSUPPORTED, "no seeded kernel for R = %d", d->lay.R);
    }
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CUDA_OK(cudaMemsetAsync(d_work, 0, kWorkBytes, st));
  if (n == 0) return SC_OK;
  DevInfo di = device_info();
  int per_sm = o.blocks_per_sm;
  if (per_sm <= 0) {
    CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k, kBlock, 0));
    if (per_sm < 1) per_sm = 1;
  }
  int64_t grid = (int64_t)di.sms * per_sm, need = (n + kBlock - 1) / kBlock;
  if (grid > need) grid = need;
  sct::Params p;
  std::memset(&p, 0, sizeof(p));
  fill_params(d, p);
  p.rays = reinterpret_cast<const float4*>(d_rays);
  p.hits = reinterpret_cast<float4*>(d_hits);
  p.counts = reinterpret_cast<uint2*>(d_counts);
  p.work = reinterpret_cast<unsigned*>(d_work);
  p.status = p.work + 1;
  p.n = n;
  p.refill = o.refill ? o.refill : kDefaultRefill;
  k<<<(unsigned)grid, kBlock, 0, st>>>(p, d_cls, reinterpret_cast<const float4*>(d_frontier),
                                       n_frontier);
  CUDA_OK(cudaGetLastError());
  return SC_OK;
  SC_CATCH
}

sc_status sc_trace_host(const sc_dbvh* d, const float* h_rays, int64_t n, sc_hit* h_hits,
                        uint32_t* h_counts, int mode, int cull, const sc_trace_opts* opts,
                        float* d_rays_buf, sc_hit* d_hits_buf, uint32_t* d_counts_buf,
                        void* d_work, size_t work_bytes, void* stream) {
  SC_TRY
  if (n > 0 && (!h_rays || !h_hits || !d_rays_buf || !d_hits_buf))
    fail(SC_ERR_ARG, "sc_trace_host: NULL buffer");
  if (h_counts && !d_counts_buf) fail(SC_ERR_ARG, "sc_trace_host: counts need d_counts_buf");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n > 0)
    CUDA_OK(cudaMemcpyAsync(d_rays_buf, h_rays, (size_t)n * 32, cudaMemcpyHostToDevice, st));
  launch_trace(d, d_rays_buf, n, d_hits_buf, h_counts ? d_counts_buf : nullptr, mode, cull, opts,
               d_work, work_bytes, st);
  if (n > 0) {
    CUDA_OK(cudaMemcpyAsync(h_hits, d_hits_buf, (size_t)n * 16, cudaMemcpyDeviceToHost, st));
    if (h_counts)
      CUDA_OK(cudaMemcpyAsync(h_counts, d_counts_buf, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
  }
  CUDA_OK(cudaStreamSynchronize(st));
  return SC_OK;
  SC_CATCH
}

sc_status sc_trace_noalloc(const sc_dbvh* d, const float* d_rays, int64_t n, sc_hit* d_hits,
                           uint32_t* d_counts, int mode, int cull, const sc_trace_opts* opts,
                           void* stream) {
  SC_TRY
  {
    // the call waits for its trace and reads the status back, which a
    // stream capture cannot record: refuse before touching the stream
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_OK(cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cs));
    if (cs != cudaStreamCaptureStatusNone)
      fail(SC_ERR_STATE, "sc_trace_noalloc cannot be captured: it waits for its trace");
  }
  const size_t need = kWorkBytes;
  if (need > kNoallocScratchBytes)
    fail(SC_ERR_UNSUPPORTED,
         "sc_trace_noalloc: the trace needs %zu bytes of scratch, the static area holds %zu", need,
         kNoallocScratchBytes);
  void* scratch = noalloc_scratch_address();
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  launch_trace(d, d_rays, n, d_hits, d_counts, mode, cull, opts, scratch, kNoallocScratchBytes,
               st);
  unsigned word[2] = {0, 0};
  CUDA_OK(cudaMemcpyAsync(word, scratch, sizeof(word), cudaMemcpyDeviceToHost, st));
  CUDA_OK(cudaStreamSynchronize(st));
  if (word[1] & sct::ST_STACK) fail(SC_ERR_STACK, "device: a traversal stack overflowed");
  if (word[1] & sct::ST_BAD_NODE)
    fail(SC_ERR_STATE, "device: the BVH image holds an invalid child reference");
  return SC_OK;
  SC_CATCH
}

size_t sc_trace_waves_workspace_bytes(int64_t n0, const sc_trace_opts* opts) {
  return waves_ws_bytes(n0, wave_chunk_of(n0, opts));
}

sc_status sc_trace_waves(const sc_dbvh* d, const float* d_rays, int64_t n0, int bounces,
                         uint32_t seed, int cull, const sc_wave_out* outs,
                         const sc_trace_opts* opts, void* d_ws, size_t ws_bytes, void* stream) {
  SC_TRY
  launch_waves(d, d_rays, n0, bounces, seed, cull, outs, opts, d_ws, ws_bytes,
               reinterpret_cast<cudaStream_t>(stream));
  return SC_OK;
  SC_CATCH
}

}  // extern "C"

namespace {

// Wave sizes and the device status of a finished wave launch (stream
// synchronized); throws on a device error.
void read_wave_sizes(const void* d_ws, int bounces, uint32_t* sizes, cudaStream_t st) {
  unsigned head[sct::WW_HEAD];
  CUDA_OK(cudaMemcpyAsync(head, d_ws, sizeof(head), cudaMemcpyDeviceToHost, st));
  CUDA_OK(cudaStreamSynchronize(st));
  const unsigned nch = head[sct::WW_NCHUNKS];
  std::vector<unsigned> cw((size_t)nch * sct::WW_CHUNK_WORDS);
  if (nch) {
    CUDA_OK(cudaMemcpyAsync(cw.data(), reinterpret_cast<const unsigned*>(d_ws) + sct::WW_HEAD,
                            cw.size() * 4, cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaStreamSynchronize(st));
  }
  for (int i = 0; i <= bounces; ++i) {
    uint64_t tot = 0;
    if (i > 0)
      for (unsigned c = 0; c < nch; ++c) tot += cw[(size_t)c * sct::WW_CHUNK_WORDS + sct::WW_SIZE + i];
    sizes[i] = (uint32_t)tot;
  }
  const unsigned status = head[sct::WW_STATUS];
  if (status & sct::ST_TIMEOUT) fail(SC_ERR_TIMEOUT, "device: a wave barrier timed out");
  if (status & sct::ST_STACK) fail(SC_ERR_STACK, "device: a traversal stack overflowed");
  if (status & sct::ST_BAD_NODE)
    fail(SC_ERR_STATE, "device: the BVH image holds an invalid child reference");
}

}  // namespace

extern "C" {

sc_status sc_trace_waves_host(const sc_dbvh* d, const float* h_rays, int64_t n0, int bounces,
                              uint32_t seed, int cull, const sc_wave_out* h_outs,
                              const sc_trace_opts* opts, float* d_rays_buf,
                              const sc_wave_out* d_outs, void* d_ws, size_t ws_bytes,
                              uint32_t* sizes, void* stream) {
  SC_TRY
  if (!h_outs || !d_outs || bounces < 0 || bounces + 1 > sct::kMaxWaves)
    fail(SC_ERR_ARG, "sc_trace_waves_host: bad arguments");
  if (n0 > 0 && (!h_rays || !d_rays_buf)) fail(SC_ERR_ARG, "sc_trace_waves_host: NULL rays");
  for (int w = 0; w <= bounces; ++w)
    if (n0 > 0 && !h_outs[w].hits)
      fail(SC_ERR_ARG, "sc_trace_waves_host: wave %d has no host hit buffer", w);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n0 > 0)
    CUDA_OK(cudaMemcpyAsync(d_rays_buf, h_rays, (size_t)n0 * 32, cudaMemcpyHostToDevice, st));
  launch_waves(d, d_rays_buf, n0, bounces, seed, cull, d_outs, opts, d_ws, ws_bytes, st);
  uint32_t local[sct::kMaxWaves] = {0};
  if (n0 > 0) read_wave_sizes(d_ws, bounces, local, st);
  local[0] = (uint32_t)n0;
  for (int w = 0; w <= bounces; ++w) {
    const size_t m = local[w];
    if (m == 0) continue;
    CUDA_OK(cudaMemcpyAsync(h_outs[w].hits, d_outs[w].hits, m * 16, cudaMemcpyDeviceToHost, st));
    if (h_outs[w].path && d_outs[w].path)
      CUDA_OK(cudaMemcpyAsync(h_outs[w].path, d_outs[w].path, m * 4, cudaMemcpyDeviceToHost, st));
    if (h_outs[w].counts && d_outs[w].counts)
      CUDA_OK(cudaMemcpyAsync(h_outs[w].counts, d_outs[w].counts, m * 8, cudaMemcpyDeviceToHost,
                              st));
    if (h_outs[w].rays && d_outs[w].rays)
      CUDA_OK(cudaMemcpyAsync(h_outs[w].rays, d_outs[w].rays, m * 32, cudaMemcpyDeviceToHost, st));
  }
  CUDA_OK(cudaStreamSynchronize(st));
  if (sizes)
    for (int w = 0; w <= bounces; ++w) sizes[w] = w == 0 ? 0u : local[w];
  return SC_OK;
  SC_CATCH
}

}  // extern "C"

extern "C" {

sc_status sc_waves_poll(const void* d_ws, int bounces, uint32_t* sizes, void* stream) {
  SC_TRY
  if (!d_ws || !sizes || bounces < 0 || bounces + 1 > sct::kMaxWaves)
    fail(SC_ERR_ARG, "sc_waves_poll: bad argument");
  read_wave_sizes(d_ws, bounces, sizes, reinterpret_cast<cudaStream_t>(stream));
  sizes[0] = 0;
  return SC_OK;
  SC_CATCH
}

sc_status sc_autotune_waves(const sc_dbvh* d, const float* d_rays, int64_t n0, int bounces,
                            uint32_t seed, int cull, const sc_wave_out* outs,
                            const sc_trace_opts* base, void* d_ws, size_t ws_bytes, int reps,
                            void* d_flush, size_t flush_bytes, sc_trace_opts* best,
                            sc_tune_result* results, int cap, int* n_results, void* stream) {
  SC_TRY
  if (!d || !best || n0 <= 0 || reps < 1) fail(SC_ERR_ARG, "sc_autotune_waves: bad argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  sc_trace_opts o{};
  o.lut_mode = SC_LUT_AUTO;
  if (base) o = *base;
  const bool all_blocks = ((!cull) || d->lay.R == 6) && o.variant == 0;
  std::vector<int> blocks = all_blocks ? std::vector<int>{64, 128, 256} : std::vector<int>{128};
  std::vector<int> stacks;
  if (all_blocks && d->stack_need <= 32) stacks.push_back(32);
  stacks.push_back(64);
  if (d->lay.width == 4) {
    blocks = {128, 256};
    stacks = {64};
  }
  const int refills[3] = {4, 8, 16};
  std::vector<int64_t> chunks = {n0};
  for (int64_t c = n0 / 2; c >= 65536 && chunks.size() < 3; c /= 2) chunks.push_back(c);
  std::vector<sc_trace_opts> cands;
  for (int blk : blocks)
    for (int stk : stacks)
      for (int rf : refills)
        for (int64_t ch : chunks) {
          sc_trace_opts t = o;
          t.block = blk;
          t.stack = stk;
          t.refill = rf;
          t.wave_chunk = ch;
          cands.push_back(t);
        }
  // the stack's top entries in a shared-memory ring, 9 resident blocks per
  // SM (56 registers a thread) and the hit's u, v and id in shared memory,
  // and their combinations: built at block 128 / stack 64 for the images
  // that have kernel variants (10 blocks per SM never won and is not tried)
  const int lutv = waves_lutv(d, o.lut_mode);
  const int placements[6] = {sct::OPT_SSTACK,
                             sct::OPT_OCC9,
                             sct::OPT_OCC9 | sct::OPT_SSTACK,
                             sct::OPT_HSLOT,
                             sct::OPT_HSLOT | sct::OPT_OCC9,
                             sct::OPT_HSLOT | sct::OPT_OCC9 | sct::OPT_SSTACK};
  if (o.variant == 0 && variant_image_ok(d, cull, lutv) && d->stack_need <= 64)
    for (int v : placements) {
      if (!sct::var_supported(v)) continue;
      for (int rf : {4, 8})
        for (int64_t ch : chunks) {
          sc_trace_opts t = o;
          t.block = kBlock;
          t.stack = sct::kStack;
          t.refill = rf;
          t.wave_chunk = ch;
          t.variant = v;
          cands.push_back(t);
        }
    }
  cudaEvent_t e0, e1;
  CUDA_OK(cudaEventCreate(&e0));
  CUDA_OK(cudaEventCreate(&e1));
  std::vector<std::vector<float>> ms(cands.size());
  auto median = [](std::vector<float> v) {
    std::sort(v.begin(), v.end());
    return v[v.size() / 2];
  };
  // one timed launch of candidate i, the flush buffer overwritten first
  auto time_one = [&](size_t i, int r) {
    if (d_flush && flush_bytes) CUDA_OK(cudaMemsetAsync(d_flush, r & 0xFF, flush_bytes, st));
    CUDA_OK(cudaEventRecord(e0, st));
    launch_waves(d, d_rays, n0, bounces, seed, cull, outs, &cands[i], d_ws, ws_bytes, st);
    CUDA_OK(cudaEventRecord(e1, st));
    CUDA_OK(cudaEventSynchronize(e1));
    float x = 0;
    CUDA_OK(cudaEventElapsedTime(&x, e0, e1));
    ms[i].push_back(x);
  };
  std::vector<size_t> order(cands.size());
  try {
    for (auto& t : cands)  // warm-up: code, first touches
      launch_waves(d, d_rays, n0, bounces, seed, cull, outs, &t, d_ws, ws_bytes, st);
    for (int r = 0; r < reps; ++r)
      for (size_t i = 0; i < cands.size(); ++i) time_one(i, r);
    // second round: candidates a few percent apart are within the run-to-run
    // spread of one launch, so the best kTop of the first round are timed
    // again, interleaved, 2 reps + 2 more times each
    std::vector<float> first(cands.size());
    for (size_t i = 0; i < cands.size(); ++i) first[i] = median(ms[i]);
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return first[a] < first[b]; });
    constexpr size_t kTop = 4;
    const size_t top = std::min(kTop, order.size());
    for (int r = 0; r < 2 * reps + 2; ++r)
      for (size_t k = 0; k < top; ++k) time_one(order[k], reps + r);
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  float best_ms = 1e30f;
  for (size_t i = 0; i < cands.size(); ++i) {
    const float med = median(ms[i]);
    if (results && (int)i < cap)
      results[i] = sc_tune_result{cands[i].block, cands[i].stack, cands[i].refill,
                                  cands[i].wave_chunk, med, cands[i].variant};
    if (med < best_ms) {
      best_ms = med;
      *best = cands[i];
    }
  }
  if (n_results) *n_results = (int)cands.size();
  return SC_OK;
  SC_CATCH
}

sc_status sc_status_poll(const void* d_work, void* stream) {
  SC_TRY
  if (!d_work) fail(SC_ERR_ARG, "sc_status_poll: NULL workspace");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned word[2] = {0, 0};
  CUDA_OK(cudaMemcpyAsync(word, d_work, sizeof(word), cudaMemcpyDeviceToHost, st));
  CUDA_OK(cudaStreamSynchronize(st));
  if (word[1] & sct::ST_STACK) {
    set_error("device: a traversal stack overflowed");
    return SC_ERR_STACK;
  }
  if (word[1] & sct::ST_BAD_NODE) {
    set_error("device: the BVH image holds an invalid child reference");
    return SC_ERR_STATE;
  }
  return SC_OK;
  SC_CATCH
}

}  // extern "C"
