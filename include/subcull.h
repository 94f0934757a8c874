/*
 * subcull.h — C-ABI of libsubcull: GB300 (sm_103a) BVH traversal with
 * subspace culling (Yoshimura & Harada, "Subspace Culling for Ray-Box
 * Intersection", 2023).
 *
 * Path: seeded scene -> binned-SAH BVH2 (Sec. 4) -> per-child object masks
 * (Sec. 3.1.1 voxelization, Sec. 3.2.1 / Alg. 2 hierarchical fill) and,
 * optionally, their compression (Sec. 3.2.2-3.2.3, Alg. 3) -> a 16-byte
 * aligned node image in device memory -> batched traversal (Alg. 4): after
 * each ray-box slab test the clipped segment is turned into a ray mask by
 * table lookup (Alg. 1) and ANDed with the child's object mask; zero culls
 * the child.
 *
 * Conventions for every entry point:
 *  - Each call returns an sc_status; on failure sc_last_error() describes
 *    it (thread-local string, valid until the next call on that thread).
 *    No C++ exception crosses this boundary.
 *  - "host" pointers are ordinary CPU memory, "device" pointers are CUDA
 *    global memory of the current device.  The library never frees memory
 *    it did not allocate; device buffers (BVH image, rays, hits, counts,
 *    workspace) belong to the caller and must outlive the work queued on
 *    the stream.  Host-side handles (sc_bvh, sc_dbvh) are owned by the
 *    library and released with the matching *_destroy call.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Device
 *    work is asynchronous; errors detected on the device (a traversal stack
 *    overflow) are recorded in the workspace and reported by
 *    sc_status_poll().
 *  - There is no CPU fallback: without a usable CUDA device the device
 *    calls return SC_ERR_CUDA.
 *
 * Layouts:
 *  - triangles: float[n][9] = v0.xyz, v1.xyz, v2.xyz (id = array index).
 *  - rays: float[n][8] = origin.xyz, tmin, direction.xyz, tmax.
 *  - hits: sc_hit[n]; a miss is {t = +inf, id = -1, u = v = 0}.
 *  - counts: uint32[n][2] = {ray-box slab tests, ray-triangle tests}.
 *  - masks: R^3 bits, bit = x + R*y + R*R*z, little-endian uint32 words,
 *    W(R) = ceil(R^3/32) words.
 */
#ifndef SUBCULL_H
#define SUBCULL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Raised whenever a struct or enum of this header changes layout or meaning.
   2: sc_tune_result gained `variant` (the autotuner also chooses the stack
   placement and the resident blocks per SM). */
#define SC_ABI_VERSION 2

typedef enum {
  SC_OK = 0,
  SC_ERR_ARG = -1,         /* invalid argument (NULL, size, range)          */
  SC_ERR_CUDA = -2,        /* a CUDA runtime call failed / no device        */
  SC_ERR_NOMEM = -3,       /* host allocation failed or buffer too small    */
  SC_ERR_TIMEOUT = -4,     /* a bounded device wait ran out                 */
  SC_ERR_STACK = -5,       /* device traversal stack overflow (recorded)    */
  SC_ERR_UNSUPPORTED = -6, /* configuration the library does not support    */
  SC_ERR_STATE = -7,       /* object in the wrong state for this call       */
  SC_ERR_IO = -8           /* file could not be read or written             */
} sc_status;

/* Message of the last failure on the calling thread ("" after success). */
const char* sc_last_error(void);
int sc_abi_version(void);

/* ------------------------------------------------------------ inputs --- */
/* Seeded synthetic scenes standing in for the paper's hair assets (Sec. 4,
   Fig. 7: Curly Hair, 12.1M thin tilted triangles). */
enum { SC_SCENE_HAIR = 0, SC_SCENE_SOUP = 1 };
typedef struct {
  int64_t count; /* hair: strands; soup: triangles                        */
  int segments;  /* hair: segments per strand (each = 2 triangles)        */
  int ground;    /* hair: append a 2-triangle quad at y = -1.2            */
} sc_scene_params;

/* Two-call size query: with tris == NULL only *n_tris is set.  tris: host
   float[cap][9].  SC_ERR_NOMEM if cap < the scene's triangle count. */
sc_status sc_scene_generate(int kind, const sc_scene_params* p, uint64_t seed,
                            float* tris, int64_t cap, int64_t* n_tris);

enum { SC_RAYS_PINHOLE = 0, SC_RAYS_RANDOM = 1 };
typedef struct {
  int width, height;    /* pinhole: image size (rays in 8x4 tile order)   */
  int64_t count;        /* random: number of rays                          */
  uint64_t jitter_seed; /* pinhole: 0 = pixel centres, else sub-pixel jitter */
} sc_ray_params;

/* Host rays: float[cap][8]; pix (host int32[cap] or NULL) receives the
   pixel index row*W+col of each pinhole ray.  Two-call size query with
   rays == NULL. */
sc_status sc_rays_generate(int kind, const sc_ray_params* p, uint64_t seed,
                           float* rays, int32_t* pix, int64_t cap,
                           int64_t* n_rays);

/* ------------------------------------------------------------- build --- */
typedef struct {
  int max_leaf;   /* triangles per leaf (1..8), default 4                   */
  int bins;       /* SAH bins per axis, default 32                          */
  int L;          /* mask approximation depth (Sec. 3.2.1), default 3       */
  int lut_size;   /* compression LUT entries (Sec. 4.4), default 256        */
  int chunk_bits; /* requirement-LUT chunk b (Sec. 3.2.3), default 8        */
  double eps_rel; /* voxel dilation / max(1, |scene coord|), default 2^-16  */
  int threads;    /* host threads, 0 = all                                  */
  int skip_bits;  /* device images: children whose (decoded) mask has at
                     least this many bits set are kept without a mask test;
                     0 = R^3 (only all-ones masks, whose test cannot fail:
                     the paper's method).  Any value gives the same hits. */
  int test_stride; /* device images: inner children are tested only at
                      depths that are multiples of this (0 or 1 = every
                      level, the paper's method); leaves are always tested */
  int leaf_min_tris; /* device images: leaf children holding fewer than this
                        many triangles are kept without a mask test (0 or 1:
                        every leaf is tested, the paper's method) */
  int gpu_masks;   /* 1: the object masks are built on the current GPU (the
                      same bits as the host build, which 0 selects); the
                      tree and the compression stay on the host.  Needs a
                      device: SC_ERR_CUDA without one. */
  int gpu_bvh;     /* 1: the binned-SAH tree is built on the current GPU:
                      the same tree (numbering, child boxes, leaf ranges,
                      triangle order; a zero bound may differ in sign) as
                      the host build, which 0 selects.  Needs bins <= 32
                      (SC_ERR_UNSUPPORTED otherwise) and a device
                      (SC_ERR_CUDA without one). */
} sc_build_opts;

void sc_build_opts_default(sc_build_opts* o);

typedef struct sc_bvh sc_bvh;

/* Builds the BVH2 (binned SAH, Sec. 4), then, when grid_res > 0, the object
   mask of every child (R = grid_res in {4, 6, 8}; Sec. 3.1.1 SAT
   voxelization and Alg. 2 from L levels below, Sec. 3.2.1), and, when
   compress != 0, the compression LUT and each child's LUT index (Sec.
   3.2.2, requirement LUTs and Alg. 3, Sec. 3.2.3).  tris: host, n <= 2^28.
   opts NULL = defaults.  *out owns copies of everything it needs. */
sc_status sc_bvh_build(const float* tris, int64_t n_tris, int grid_res,
                       int compress, const sc_build_opts* opts, sc_bvh** out);
void sc_bvh_destroy(sc_bvh* b);

typedef struct {
  int64_t num_tris, num_nodes;
  int max_depth;      /* deepest slot below the root (root = 0)           */
  int grid_res, compress, L, clut_entries;
  double eps;         /* absolute voxel dilation                           */
  float root_box[6];
  double ms_bvh, ms_masks, ms_compress; /* host build times               */
} sc_bvh_info;
sc_status sc_bvh_get_info(const sc_bvh* b, sc_bvh_info* info);

/* Copies the host arrays of the built BVH (for checkers).  Any output may
   be NULL.  root2 = {child, count} of the root slot; child/count: int32
   [num_nodes][2] (count > 0: leaf of `count` triangles starting at position
   `child` of perm; count == 0: inner node `child`); box: float
   [num_nodes][2][6] (lo.xyz, hi.xyz); perm: int32[num_tris] triangle id at
   each leaf position; masks: uint32[num_nodes][2][W]; clut:
   uint32[clut_entries][W]; cidx: uint8[num_nodes][2]. */
sc_status sc_bvh_export(const sc_bvh* b, int32_t* root2, int32_t* child,
                        int32_t* count, float* box, int32_t* perm,
                        uint32_t* masks, uint32_t* clut, uint8_t* cidx);

/* Checkpoint of a built BVH (everything sc_bvh_build computed, so that a
   large build is paid once; not in the paper).  sc_bvh_save writes `path`
   (through a temporary file renamed into place); sc_bvh_load returns a new
   handle owned by the caller (free with sc_bvh_destroy).  The file carries
   a format version, a byte-order mark and a hash; a file that fails any
   check, or whose tree indices are out of range, gives SC_ERR_IO. */
sc_status sc_bvh_save(const sc_bvh* b, const char* path);
sc_status sc_bvh_load(const char* path, sc_bvh** out);

/* Refit for moved triangles (dynamic scenes, whose mask updates the paper
   leaves to future work).  tris: host float[n_tris][9], the new positions
   of the same triangles in input order (n_tris must equal the build's).
   The topology and triangle order are kept; triangles whose coordinates
   changed (bit for bit) make every slot above them dirty; those slots'
   boxes are refit bottom-up (unions of triangle boxes, as the build takes
   them) and their object masks are computed again (on the GPU when the
   build used gpu_masks), and compressed BVHs encode them again (Alg. 3)
   against the LUT chosen at build time.  A change of the scene's dilation
   eps makes every slot dirty.  The masks then equal a mask build from
   scratch on the refit tree.  Device images are not touched: upload again.
   info (may be NULL) receives the counts and timings.  SC_ERR_ARG for a
   NULL bvh, another triangle count or a non-finite coordinate. */
typedef struct {
  int64_t moved_tris;   /* triangles whose coordinates changed            */
  int64_t dirty_nodes;  /* nodes whose boxes / masks were computed again  */
  double ms_boxes, ms_masks, ms_compress;
} sc_refit_info;
sc_status sc_bvh_refit(sc_bvh* b, const float* tris, int64_t n_tris, sc_refit_info* info);

/* The ray-mask table (Sec. 3.1.1): uint32[R^3 * R^3][W], row
   beg*R^3 + end, cell index x + R*y + R*R*z.  Built here from the 2-D
   sweep tables of each pair of axes (Helly's theorem on intervals of t). */
sc_status sc_raylut(int R, uint32_t* lut);

/* The ray-mask table at R_ray = 2R (Sec. 4.2), R in {2, 3, 4, 6}:
   uint32[(2R)^6][W] (W = words of an R^3-bit mask), row beg*(2R)^3 + end
   with beg, end cells x + 2R*y + 4R^2*z of the 2R grid; mask cell v is set
   iff the sweep test on the 2R grid sets one of v's eight sub-cells (each
   2R cell lies in one mask cell).  The caller owns lut; SC_ERR_ARG for
   another R or a NULL lut. */
sc_status sc_raylut2r(int R, uint32_t* lut);

/* ------------------------------------------------------ device image --- */
enum {
  SC_LAYOUT_PLAIN = 0,         /* 64-B nodes without masks (unculled baseline) */
  SC_LAYOUT_MASKED = 1,        /* masks (or LUT indices) plus each child's
                                  Alg. 1 scales R/extent precomputed in the
                                  node: 96 B compressed, 64+32+2*mask bytes
                                  uncompressed, rounded up to a multiple of
                                  32 B (128 / 160 / 224 B at R = 4 / 6 / 8) */
  SC_LAYOUT_PLAIN4 = 3,        /* 4-wide nodes without masks (see below)         */
  SC_LAYOUT_MASKED4 = 4,       /* 4-wide nodes with masks (or LUT indices) and
                                  scales.  4-wide nodes (the paper's Sec. 3.2.4
                                  setting): the node made from binary node n
                                  holds, in order, for each child slot c of n,
                                  the two child slots of c if c is inner, else
                                  c itself (2..4 children, each keeping its
                                  binary slot's box, mask and LUT index);
                                  pre-order numbering.  Record: six float4 of
                                  lo.x, lo.y, lo.z, hi.x, hi.y, hi.z of the
                                  four children, the four slot words (unused:
                                  0xFFFFFFFF), the four meta words, then (masked)
                                  the four children's scales as three float4
                                  and, from byte 192, the four masks: 128
                                  bytes plain, 176 compressed, 192 + 4 mask
                                  strides else.
                                  Children are visited by entry distance,
                                  ties by position. */
  SC_LAYOUT_MASKED_COMPACT = 2, /* masks (or LUT indices) only; the scales are
                                  divided on the fly: 64 B compressed,
                                  64+2*mask bytes uncompressed, rounded up to
                                  a multiple of 32 B (96 / 128 / 192 B)      */
  SC_LAYOUT_MASKED_RAY2R = 5   /* SC_LAYOUT_MASKED plus the ray-mask table at
                                  R_ray = 2R (Sec. 4.2): begin and end cells
                                  on the 2R grid (twice the R-grid coordinate,
                                  rounded down), one R^3-bit row per pair, a
                                  mask cell set iff the sweep test on the 2R
                                  grid sets one of its eight sub-cells;
                                  (2R)^6 rows: 2 MB at R = 4, 96 MB at R = 6.
                                  Uncompressed masks, R = 4 or 6 only
                                  (SC_ERR_UNSUPPORTED otherwise).           */
};

/* Bytes of the device image of `b` in `layout` (a multiple of 256). */
sc_status sc_bvh_device_bytes(const sc_bvh* b, int layout, size_t* nbytes);

typedef struct sc_dbvh sc_dbvh;

/* Packs the image on the host and copies it (cudaMemcpyAsync on `stream`)
   into d_buf: device memory of >= nbytes bytes, 256-byte aligned, owned by
   the caller.  The image holds 16-B aligned nodes (fetched with 128-bit
   loads), 48-B triangles {v0,id}{e1}{e2} in leaf order, the ray-mask
   tables, the compression LUT and (compressed) the bit table of every ray
   mask against every LUT entry.  *out is a host-side view of d_buf;
   destroying it does not touch d_buf. */
sc_status sc_bvh_upload(const sc_bvh* b, int layout, void* d_buf, size_t nbytes,
                        void* stream, sc_dbvh** out);
void sc_dbvh_destroy(sc_dbvh* d);

/* ------------------------------------------------------------- trace --- */
typedef struct {
  float t;
  int32_t id;
  float u, v;
} sc_hit;

enum { SC_CLOSEST = 0, SC_ANY = 1 };

enum { SC_LUT_AUTO = 0, SC_LUT_GLOBAL = 1, SC_LUT_SHARED = 2, SC_LUT_BITTABLE = 3,
       SC_LUT_RAY2R = 4, SC_LUT_FACTORED_L1 = 5 };

typedef struct {
  int block;         /* threads per block: 0 (= 128) or 128               */
  int blocks_per_sm; /* persistent blocks per SM, 0 = occupancy maximum    */
  int lut_mode;      /* ray-mask lookup: SC_LUT_GLOBAL = full table through
                        L1/L2; SC_LUT_SHARED = shared memory (R = 4: the
                        whole 32-KB table and the LUT; R = 6, 8: factored
                        per-axis-pair tables in single-batch traces, and
                        in the wave pipeline for R = 6 uncompressed images
                        with stored scales; other wave launches and
                        seeded traces use the full table);
                        SC_LUT_BITTABLE (compressed images) = the
                        precomputed bit table of Sec. 3.2.2, one bit per
                        (ray mask, LUT entry); SC_LUT_RAY2R (images in
                        SC_LAYOUT_MASKED_RAY2R) = the R_ray = 2R table;
                        SC_LUT_FACTORED_L1 = the factored tables read from
                        the image through L1 (binary R = 6 uncompressed
                        images with stored scales; seeded traces use the
                        full table), else SC_ERR_UNSUPPORTED;
                        SC_LUT_AUTO = the 2R table when the image holds it,
                        else the bit table when compressed, else the full
                        table                                             */
  int refill;        /* a warp fetches new rays once this many of its lanes
                        are idle (1..32), 0 = default                     */
  int stack;         /* waves: traversal stack entries, 32 or 64 (0 = 64)  */
  int64_t wave_chunk;/* waves: primary rays per chunk (the wave size); each
                        chunk runs through all its bounce waves before the
                        next; 0 = all primary rays in one chunk           */
  int64_t wait_timeout_ns; /* waves: limit of each device-wide wait (the
                        barrier between waves), 0 = 2 s.  A wait that runs
                        out records SC_ERR_TIMEOUT, which sc_waves_poll
                        returns, and the kernel returns; the context stays
                        usable.                                           */
  int variant;       /* kernel options, a bit field of SC_VARIANT_* (0 =
                        the defaults).  Built for R = 6 images (uncompressed
                        with the full table, compressed with the bit
                        table) and the plain traversal, in sc_trace and,
                        with block 128 / stack 64, sc_trace_waves; other
                        combinations give SC_ERR_UNSUPPORTED.             */
} sc_trace_opts;

/* Kernel options of sc_trace_opts.variant.  Only SC_VARIANT_FUSED_CELLS
   changes results: it evaluates the Alg. 1 cell coordinate in the ray
   parameter as one fused multiply-add, s (o - lower) + t (s d) with
   s = R / extent, instead of the paper's order (p = o + t d, then
   s (p - lower)); cells can then differ where the coordinate lies within
   rounding of a cell border (the object masks' dilation keeps culling
   conservative).  The others change only the timing of loads, where the
   top stack entry lives and the order in which bounce rays are traced; hits
   and per-ray counts are unchanged. */
enum {
  SC_VARIANT_FUSED_CELLS = 1,  /* fused Alg. 1 coordinate (see above)        */
  SC_VARIANT_PAIR = 2,         /* both children's lookups in flight together */
  SC_VARIANT_SPEC = 4,         /* the nearer child's record requested before
                                  the culling results arrive                */
  SC_VARIANT_TOS = 8,          /* top stack entry held in registers          */
  SC_VARIANT_SORT = 16,        /* waves: bounce queues sorted by direction
                                  octant and origin cell before tracing     */
  SC_VARIANT_LAZY = 64,        /* the per-child Alg. 1 scales are fetched only
                                  for nodes with a child to test            */
  SC_VARIANT_SSTACK = 128,     /* the top 8 stack entries of each ray in
                                  shared memory, the rest in local memory   */
  SC_VARIANT_TABLE_L1 = 256,   /* rows of the full ray-mask table (R = 6,
                                  8) and of the R_ray = 2R table, and the
                                  uncompressed object masks, allocated in
                                  L1 like other loads; by default they are
                                  loaded without L1 allocation, so that
                                  they do not evict node records            */
  SC_VARIANT_OCC9 = 1024,      /* waves: 9 resident blocks of 128 threads per
                                  SM (56 registers a thread) instead of 8
                                  (64 registers); combinable with
                                  SC_VARIANT_SSTACK                         */
  SC_VARIANT_OCC10 = 2048,     /* waves: 10 resident blocks per SM (48
                                  registers); combinable with
                                  SC_VARIANT_SSTACK                         */
  SC_VARIANT_HSLOT = 4096,     /* the accepted hit's u, v and triangle id in
                                  a per-thread shared-memory slot instead of
                                  registers; combinable with SC_VARIANT_OCC9
                                  and SC_VARIANT_SSTACK                     */
  SC_VARIANT_DEFER = 32        /* compressed masks with the bit table: each
                                  child's bit-table lookup is issued when the
                                  child is visited, beside its own fetch
                                  (its cells still come from the parent's
                                  slab test); other images ignore the bit    */
};

/* Workspace bytes sc_trace needs (ray counter and device status word). */
size_t sc_trace_workspace_bytes(void);

/*
 * Traces n rays (Alg. 4).  d_rays: device float[n][8]; d_hits: device
 * sc_hit[n]; d_counts: device uint32[n][2] or NULL.  mode SC_CLOSEST or
 * SC_ANY.  cull != 0 applies subspace culling (Sec. 3.1.2): the image must
 * be SC_LAYOUT_MASKED[_COMPACT] with grid_res > 0; cull == 0 runs the plain traversal
 * on any layout.  d_work: device workspace of >= sc_trace_workspace_bytes()
 * bytes (reset by this call).  Asynchronous on `stream`.
 */
sc_status sc_trace(const sc_dbvh* d, const float* d_rays, int64_t n,
                   sc_hit* d_hits, uint32_t* d_counts, int mode, int cull,
                   const sc_trace_opts* opts, void* d_work, size_t work_bytes,
                   void* stream);

/*
 * End-to-end form of sc_trace for host data: copies h_rays (host float
 * [n][8], ideally pinned) to d_rays_buf, traces, and copies the hits (and
 * counts if h_counts != NULL) back to h_hits / h_counts, all on `stream`,
 * then synchronizes it.  d_rays_buf, d_hits_buf, d_counts_buf: device
 * scratch of n*32, n*16 and n*8 bytes owned by the caller.
 */
sc_status sc_trace_host(const sc_dbvh* d, const float* h_rays, int64_t n,
                        sc_hit* h_hits, uint32_t* h_counts, int mode, int cull,
                        const sc_trace_opts* opts, float* d_rays_buf,
                        sc_hit* d_hits_buf, uint32_t* d_counts_buf,
                        void* d_work, size_t work_bytes, void* stream);

/*
 * sc_trace for callers that cannot allocate device memory.  Some hosts own
 * all of the GPU's memory through their own allocator (a renderer or a
 * framework with a caching pool) and fail or stall on an extra cudaMalloc,
 * which may also synchronize the whole device; such callers cannot create
 * the workspace sc_trace takes.  This entry point allocates nothing: the
 * ray counter and status word live in a static device array of 256 bytes
 * that every GPU loading this library holds until exit.  (The paper has no
 * counterpart: this is an interface convenience.)
 *
 * Arguments as for sc_trace, without the workspace: the caller still passes
 * the image, rays, hits and (optional) counts.  The call clears the scratch,
 * launches the trace on `stream`, waits for it and returns the device
 * status (SC_ERR_STACK / SC_ERR_STATE as sc_status_poll would); every call
 * blocks until its trace has finished.  The first call on a device looks up
 * the array's device address (once per device, with that device current)
 * and keeps it for the life of the process, so the library must not be used
 * across a cudaDeviceReset.  No call can be captured in a CUDA graph (each
 * one waits for its trace): on a capturing stream the call returns
 * SC_ERR_STATE before it enqueues anything, and the capture stays valid.
 * All calls share the one array, which keeps the last call's
 * contents: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialized by the caller.  Returns
 * SC_ERR_UNSUPPORTED if the trace ever needed more scratch than the array
 * holds; no cudaMalloc, cudaFree or allocating library routine is called.
 */
sc_status sc_trace_noalloc(const sc_dbvh* d, const float* d_rays, int64_t n,
                           sc_hit* d_hits, uint32_t* d_counts, int mode,
                           int cull, const sc_trace_opts* opts, void* stream);

/* ------------------------------------------------------------- waves --- */
/* Primary rays plus diffuse bounce waves in one persistent (cooperative)
   launch.  The paper's workload is path tracing (Sec. 4); here every
   closest hit of wave w spawns one cosine-weighted bounce ray (random bits
   from the hash of Jarzynski & Olano 2020 keyed by seed, path id and
   bounce) into the queue of wave w+1, so later waves hold only spawned
   rays; a bounded grid barrier separates the waves.  Capturable in a CUDA
   graph (the launch is a cooperative kernel node). */
#define SC_MAX_BOUNCES 4

typedef struct {
  sc_hit* hits;     /* device sc_hit[n0]: wave entries in queue order      */
  int32_t* path;    /* device int32[n0] or NULL: primary ray of each entry */
  uint32_t* counts; /* device uint32[n0][2] or NULL                        */
  float* rays;      /* device float[n0][8] or NULL: the traced rays         */
} sc_wave_out;

/* Workspace bytes sc_trace_waves needs for n0 primary rays with opts'
   wave_chunk (NULL = one chunk): two ray queues of one chunk and their path
   ids, a third queue and a 32,768-entry histogram for the bounce-queue sort
   (SC_VARIANT_SORT), and the control words. */
size_t sc_trace_waves_workspace_bytes(int64_t n0, const sc_trace_opts* opts);

/* d_rays: device float[n0][8] primary rays; outs: host array of bounces+1
   sc_wave_out (each buffer sized for n0 entries); d_ws: device workspace,
   256-byte aligned, >= sc_trace_waves_workspace_bytes(n0); cull as in
   sc_trace (closest hit only).  Asynchronous; wave sizes and the device
   status come from sc_waves_poll. */
sc_status sc_trace_waves(const sc_dbvh* d, const float* d_rays, int64_t n0,
                         int bounces, uint32_t seed, int cull,
                         const sc_wave_out* outs, const sc_trace_opts* opts,
                         void* d_ws, size_t ws_bytes, void* stream);

/* Synchronizes `stream`; sizes (host uint32[bounces+1]) receives the number
   of rays of each bounce wave (sizes[0] = 0: wave 0 is the n0 primaries).
   Returns SC_ERR_TIMEOUT / SC_ERR_STACK / SC_ERR_STATE on device errors. */
sc_status sc_waves_poll(const void* d_ws, int bounces, uint32_t* sizes, void* stream);

/* End-to-end form of sc_trace_waves for host data: copies h_rays (host
   float[n0][8], ideally pinned) to d_rays_buf (device, n0 * 32 bytes,
   16-byte aligned), runs the wave pipeline into the device buffers d_outs
   (as sc_trace_waves), reads the wave sizes, and copies each wave's entries
   back to the host buffers h_outs: hits always (h_outs[w].hits: host
   sc_hit[n0]), path ids, counts and traced rays where both the host and the
   device pointer are given; then synchronizes `stream`.  sizes (host
   uint32[bounces+1] or NULL) as sc_waves_poll.  Device errors as
   sc_waves_poll. */
sc_status sc_trace_waves_host(const sc_dbvh* d, const float* h_rays, int64_t n0, int bounces,
                              uint32_t seed, int cull, const sc_wave_out* h_outs,
                              const sc_trace_opts* opts, float* d_rays_buf,
                              const sc_wave_out* d_outs, void* d_ws, size_t ws_bytes,
                              uint32_t* sizes, void* stream);

/* Autotuner of the wave pipeline: times sc_trace_waves (one warm-up, then
   `reps` rounds over all candidates, then 2 reps + 2 more rounds over the
   four fastest of them, CUDA events, median per candidate over all its
   runs;
   when d_flush is not NULL its flush_bytes -- make it larger than the L2
   cache -- are overwritten before every timed run, so candidates are
   compared from a cold cache) for block size {64, 128, 256},
   stack depth {32, 64} (where the BVH fits), refill {4, 8, 16} and wave
   chunk {n0, n0/2, n0/4} (chunks of at least 65,536 rays), writes the
   fastest into *best (block, stack, refill and wave_chunk set; other fields
   from `base`), and the tried configurations into results (host array of
   `cap` entries, may be NULL) with their count in *n_results.  Block sizes
   other than 128 and stack 32 exist for R = 6 and plain traversal only.
   When base->variant is 0 and the image has kernel variants, the candidates
   also hold block 128 / stack 64 (refill 4 and 8) with SC_VARIANT_SSTACK
   (the top stack entries in shared memory), SC_VARIANT_OCC9 (more resident
   blocks, fewer registers), SC_VARIANT_HSLOT (the hit's u, v and id in
   shared memory) and their combinations; *best->variant then says which
   was chosen.
   d_ws must be sized for the largest chunk (wave_chunk = 0).  Synchronous. */
typedef struct {
  int block, stack, refill;
  int64_t wave_chunk;
  float ms;
  int variant;  /* SC_VARIANT_SSTACK for the shared-memory stack ring, else 0 */
} sc_tune_result;

sc_status sc_autotune_waves(const sc_dbvh* d, const float* d_rays, int64_t n0,
                            int bounces, uint32_t seed, int cull,
                            const sc_wave_out* outs, const sc_trace_opts* base,
                            void* d_ws, size_t ws_bytes, int reps,
                            void* d_flush, size_t flush_bytes,
                            sc_trace_opts* best, sc_tune_result* results,
                            int cap, int* n_results, void* stream);

/* --------------------------------------------------- learned proposal --- */
/* Not in the paper.  A small network proposes, per ray, the depth-`depth`
   subtree of the BVH most likely to hold the closest hit; that subtree is
   traced first, and its hit t (if any) tightens t_max of the full culled
   traversal that follows, so results are exactly those of the traversal
   without the proposal.

   Frontier: the slots at depth `depth` below the root (the root slot has
   depth 0), plus leaf slots reached before that depth, in pre-order (left
   child first); at most 2^depth entries, 32 bytes each: the slot's box as
   its parent stores it (the scene box for the root slot) and its slot word
   (an inner node index, or 0x80000000 | (count-1) << 28 | first triangle
   position). */
typedef struct {
  float lo[3], hi[3];
  uint32_t slot;
  uint32_t reserved; /* 0 */
} sc_frontier_entry;

/* out: host sc_frontier_entry[cap]; *n_slots <- the number written;
   class_of_tri: host uint8[num_tris] or NULL, the frontier index of each
   triangle id.  depth 0..8.  SC_ERR_NOMEM if cap is too small. */
sc_status sc_bvh_frontier(const sc_bvh* b, int depth, sc_frontier_entry* out, int cap,
                          int* n_slots, uint8_t* class_of_tri);

/* Seeded traversal (closest hit).  d_cls: device int32[n], the proposed
   frontier index of each ray; an index outside [0, n_frontier) traces that
   ray without a seed.  d_frontier: device sc_frontier_entry[n_frontier]
   (16-byte aligned), n_frontier 1..256.  For a seeded ray the seed box is
   slab-tested with the ray's t_max (one node test); if the ray enters it,
   phase 1 traverses the seed subtree with that t_max.  Phase 2 traverses
   from the root, skipping the seed slot: a phase-1 hit at t_s is held
   provisionally with t_max = nextafter(t_s, +inf), and t_max drops to t_s
   when phase 2 reaches the seed slot in its traversal order, so hits are
   bit-identical to sc_trace's closest hits; counts (node tests, triangle
   tests) sum both phases.  Other arguments as sc_trace (block and stack
   must be default). */
sc_status sc_trace_seeded(const sc_dbvh* d, const float* d_rays, int64_t n,
                          const int32_t* d_cls, const sc_frontier_entry* d_frontier,
                          int n_frontier, sc_hit* d_hits, uint32_t* d_counts,
                          int cull, const sc_trace_opts* opts, void* d_work,
                          size_t work_bytes, void* stream);

/* The network: MLP 6 -> 64 -> 64 -> 256, GELU, BF16 weights, FP32
   accumulation.  Input of a ray: (origin - box centre) / box half-extent
   and the direction; d_box: device float[6] = centre.xyz, half.xyz.
   Parameters: sc_mlp_num_params() floats, layout W1[64][6], b1[64],
   W2[64][64], b2[64], W3[256][64], b3[256]; d_wb: the BF16 copy (2 bytes
   per parameter) that the kernels read. */
int sc_mlp_num_params(void);
/* d_wb <- BF16(d_w) (round to nearest even). */
sc_status sc_mlp_to_bf16(const float* d_w, void* d_wb, void* stream);
/* Top-1 class of each ray (d_cls: device int32[n]) and optionally all
   logits (d_logits: device float[n][256] or NULL).  With min_prob > 0 a
   ray whose top-1 softmax probability is below min_prob gets class -1
   (no seed: sc_trace_seeded then traces it plainly). */
sc_status sc_mlp_forward(const void* d_wb, const float* d_rays, int64_t n,
                         const float* d_box, int32_t* d_cls, float* d_logits,
                         float min_prob, void* stream);
/* The same top-1 / logits on the tensor cores: layers 2 and 3 run as
   tcgen05 BF16 x BF16 -> FP32 matrix products over tiles of 128 rays, with
   the hidden activations rounded to BF16 on entry (layer 1 and the
   epilogues in FP32).  d_status: device uint32, set to 0 by the call and to
   a non-zero value if a wait for the tensor cores ran out (the kernel then
   stops early; poll it after synchronizing).  Logits agree with
   sc_mlp_forward to the BF16 rounding of the activations. */
sc_status sc_mlp_forward_tc(const void* d_wb, const float* d_rays, int64_t n,
                            const float* d_box, int32_t* d_cls, float* d_logits,
                            float min_prob, void* d_status, void* stream);
/* Workspace bytes of one training batch. */
size_t sc_mlp_train_workspace_bytes(int64_t batch);
/* Gradient of the mean cross-entropy of a batch (d_labels: int32 classes)
   w.r.t. the parameters, ADDED to d_grad (float[P]); *d_loss (device) <-
   the mean loss.  Forward with the BF16 weights, FP32 accumulation. */
sc_status sc_mlp_grad(const void* d_wb, const float* d_rays, const int32_t* d_labels,
                      int64_t batch, const float* d_box, float* d_grad, float* d_loss,
                      void* d_ws, size_t ws_bytes, void* stream);
/* The same gradient and loss with the contractions on the tensor cores
   (tcgen05, BF16 operands, FP32 accumulation in tensor memory): the
   forward's layers 2 and 3 (hidden activations rounded to BF16, as in
   sc_mlp_forward_tc), the weight gradients dW += dA^T H over split-K batch
   slices (with a column of ones for the bias gradient), and the hidden
   backward (dA W) * gelu'(A).  Every operand of a product is rounded to BF16
   (dZ, dA, the activations and features); softmax, GELU and its derivative
   run in FP32.  d_status: device uint32 that the caller zeroes; a call ORs
   a non-zero value into it if a wait for the tensor cores ran out (the
   kernels then stop early), so one check after many steps covers them all.
   Same workspace as sc_mlp_grad. */
sc_status sc_mlp_grad_tc(const void* d_wb, const float* d_rays, const int32_t* d_labels,
                         int64_t batch, const float* d_box, float* d_grad, float* d_loss,
                         void* d_ws, size_t ws_bytes, void* d_status, void* stream);
/* Adam step `step` (1-based) on the FP32 master d_w with d_grad (then
   zeroed), moments d_m, d_v; refreshes d_wb. */
sc_status sc_mlp_adam(float* d_w, void* d_wb, float* d_grad, float* d_m, float* d_v,
                      int step, float lr, float beta1, float beta2, float eps,
                      void* stream);
/* Minibatch gather for training, shuffled on the device: d_out_rays[i] /
   d_out_labels[i] <- row perm(start + i) of d_rays (device float[n][8],
   16-byte aligned) / d_labels (device int32[n]) for i < batch, where perm is
   a pseudo-random permutation of [0, n) chosen by `key` (a 4-round Feistel
   network on the smallest domain of an even number of bits holding n, with
   cycle walking into [0, n)).  Batches start, start + batch, ... of one key
   cover an epoch without repeats.  SC_ERR_ARG unless 0 <= start and
   start + batch <= n < 2^31. */
sc_status sc_mlp_gather(const float* d_rays, const int32_t* d_labels, int64_t n,
                        uint64_t key, int64_t start, int64_t batch, float* d_out_rays,
                        int32_t* d_out_labels, void* stream);
/* Training pairs: appends (ray, class_of_tri[hit id]) of every ray that hit
   to d_out_rays / d_out_labels at position atomicAdd(d_count); at most cap. */
sc_status sc_mlp_labels(const float* d_rays, const void* d_hits, int64_t n,
                        const uint8_t* d_class_of_tri, float* d_out_rays,
                        int32_t* d_out_labels, uint32_t* d_count, int64_t cap,
                        void* stream);

/* Synchronizes `stream` and returns the device status word of d_work
   (SC_OK, or SC_ERR_STACK if a ray's stack overflowed). */
sc_status sc_status_poll(const void* d_work, void* stream);

/* ------------------------------------------------ L2 bandwidth probe --- */
/* The roofline denominator for work whose data stays in L2 (not in the
   paper).  sc_l2_read launches sc_l2_probe_blocks() blocks on `stream` that
   read the bytes at d_buf (device, 16-byte aligned, a non-zero multiple of
   16 bytes) `reps` times through L2 only (no L1 allocation), each block
   XOR-folding the 32-bit words it read into d_sink[block] (device uint64,
   at least sc_l2_probe_blocks() entries; with an odd reps the XOR of all
   sinks is the XOR of the buffer's words).  Time it with events on the
   stream; bytes * reps were read.  SC_ERR_ARG for a NULL or misaligned
   buffer or reps < 1, SC_ERR_CUDA without a device.  sc_l2_probe_blocks
   returns 0 without a device. */
int sc_l2_probe_blocks(void);
sc_status sc_l2_read(const void* d_buf, size_t bytes, int reps, uint64_t* d_sink,
                     void* stream);

#ifdef __cplusplus
}
#endif
#endif
