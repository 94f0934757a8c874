/*
 * oracle.h — plain CPU oracle for BVH traversal with subspace culling
 * (Yoshimura & Harada, "Subspace Culling for Ray-Box Intersection", 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is a slow, direct restatement of
 * the paper's definitions and algorithms.  It exists so that tests, the
 * package's smoke check and the benchmark's CPU baseline can check and time
 * the GPU path against it.  The product never links it, and it shares no
 * code or header with the product.
 *
 * Conventions (shared *by specification* with the GPU path, not by code):
 *  - triangles: float[n][9] (v0, v1, v2); the id of a triangle is its index.
 *  - rays: float[n][8] = o.xyz, tmin, d.xyz, tmax.
 *  - voxel bit order inside an R^3 mask: bit = x + R*y + R*R*z, packed in
 *    little-endian uint32 words; W(R) = ceil(R^3 / 32) words per mask.
 *  - BVH: binary, nodes hold two child slots; slot (child, count): count > 0
 *    is a leaf with `count` triangles starting at position `child` of the
 *    permuted triangle order, count == 0 an inner node with index `child`.
 *    Node 0 is the root's node; nodes are numbered in pre-order.
 */
#ifndef SUBCULL_ORACLE_H
#define SUBCULL_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int or_mask_words(int R);

/* Ray-mask lookup table (Sec. 3.1.1): bit v of entry (beg, end) is set iff
   cell v is met by the sweep of cell beg towards cell end. */
int or_raylut_cell(int R, const int* b, const int* e, const int* v);
void or_raylut(int R, uint32_t* lut /* [R^3 * R^3][W] */);
/* R_ray = 2R table (Sec. 4.2): rows [row_begin, row_end) of [(2R)^6][W]. */
void or_raylut2r_rows(int R, int64_t row_begin, int64_t row_end, uint32_t* lut);
int or_cell2_t(float t, float o, float d, float lo, float hi, int R);
int or_cell2_at(float t, float o, float d, float lo, float hi, int R, int form);

/* Conservative voxelization (Sec. 3.1.1): triangle-box overlap by the
   separating axis theorem, in double. */
int or_tri_box(const double* tri9, const double* bmin, const double* bmax);
void or_voxelize(const float* tri9, const float* lo, const float* hi, int R,
                 double eps, uint32_t* mask);
/* Hierarchical fill (Alg. 2), borders dilated by eps. */
void or_fill(uint32_t* mask, const float* plo, const float* phi,
             const uint32_t* cmask, const float* clo, const float* chi, int R,
             double eps);

/* Compression LUT (Sec. 3.2.2, 3.2.3). */
int or_clut_build(const uint32_t* masks, const float* boxes, int64_t nslots,
                  int R, int K, uint32_t* clut /* [K][W] */,
                  double* importance /* [K] or NULL */);
void or_req_luts(const uint32_t* clut, int K, int R, int b,
                 uint32_t* req /* [ceil(R^3/b)][2^b][8] */);
int or_encode(const uint32_t* mask, const uint32_t* req, int R, int b);
int or_encode_naive(const uint32_t* mask, const uint32_t* clut, int K, int R);

/* BVH (binned SAH, binary) + masks + compression. */
typedef struct OrBvh OrBvh;
OrBvh* or_bvh_build(const float* tris, int64_t n, int max_leaf, int bins);
void or_bvh_free(OrBvh* b);
/* 1: every later culling test of this BVH uses the exact ray mask (the
   cells the clipped segment meets, found in double) instead of the
   lookup table -- the paper's "ideal culling" reference of Sec. 4.1. */
void or_bvh_set_ideal(OrBvh* b, int ideal);
/* Threads of the build (the tree's independent subtrees, the masks of one
   depth level, the LUT encodings): 0 = every online core; task_tris = the
   largest range built as one subtree task (0: automatic).  The results do
   not depend on either. */
void or_set_threads(int threads, int64_t task_tris);
/* Alg. 1 cell form of the culling tests: 0 = as written, p = o + t d then
   floor(R/extent * (p - lower)) (default); 1 = the fused form of
   or_cell_t, an option of the GPU traversal mirrored here. */
void or_bvh_set_cellform(OrBvh* b, int form);
/* Refit: slot boxes from moved triangles, topology kept (masks: or_bvh_masks). */
int or_bvh_refit(OrBvh* b, const float* tris);
/* Alg. 3 for every slot against the existing compression LUT. */
int or_bvh_reencode(OrBvh* b);
/* Culling tests look up the R_ray = 2R table (caller-owned; NULL: off). */
void or_bvh_set_raylut2r(OrBvh* b, const uint32_t* lut2r);
int64_t or_bvh_num_nodes(const OrBvh* b);
int or_bvh_max_depth(const OrBvh* b);
void or_bvh_root(const OrBvh* b, int32_t* child, int32_t* count, float* box6);
void or_bvh_nodes(const OrBvh* b, int32_t* child, int32_t* count, float* box);
void or_bvh_perm(const OrBvh* b, int32_t* perm);
double or_bvh_sah(const OrBvh* b, double ct, double ci);
double or_scene_eps(const float* tris, int64_t n, double eps_rel);
int or_bvh_masks(OrBvh* b, const float* tris, int R, int L, double eps);
void or_bvh_get_masks(const OrBvh* b, uint32_t* masks /* [nn][2][W] */);
int or_bvh_compress(OrBvh* b, int K, int bits);
void or_bvh_get_clut(const OrBvh* b, uint32_t* clut, uint8_t* idx);

/* Traversal (Alg. 4 with Alg. 1).  mode 0 = closest hit, 1 = any hit.
   cull: 0 = plain, 1 = uncompressed masks, 2 = compressed masks.
   hit_t/hit_id/hit_uv: n, n, 2n; counts: [n][2] {node tests, tri tests};
   mask_tests: n or NULL.  Returns 0 or a negative error. */
int or_trace(const OrBvh* b, const float* tris, const float* rays, int64_t n,
             int mode, int cull, float* hit_t, int32_t* hit_id, float* hit_uv,
             uint32_t* counts, uint32_t* mask_tests);
/* The same, for rays [r_begin, r_end) only (threads may split the rays).
   Test selection: children whose mask has >= skip_bits bits set are kept
   untested (R^3: only all-ones masks), and inner children are tested only
   at depths that are multiples of `stride` (1: every level), and leaf
   children with fewer than leaf_min triangles are kept untested.  skip_bits
   = R^3, stride = 1 and leaf_min <= 1 is the paper's method. */
int or_trace_range(const OrBvh* b, const float* tris, const float* rays,
                   int64_t r_begin, int64_t r_end, int mode, int cull,
                   int skip_bits, int stride, int leaf_min, float* hit_t, int32_t* hit_id,
                   float* hit_uv, uint32_t* counts, uint32_t* mask_tests);

/* Brute force over all ray x triangle pairs, same ray-triangle test.
   t2: second smallest accepted t (or +inf), for near-tie detection. */
void or_brute(const float* tris, int64_t ntri, const float* rays, int64_t n,
              int mode, float* hit_t, int32_t* hit_id, float* t2);

/* Diffuse bounce rays of the wave workloads (not in the paper): counter-based
   hash (Jarzynski & Olano 2020) and a cosine-weighted direction about the
   geometric normal.  Returns 0 (no ray) for a degenerate triangle. */
uint32_t or_pcg_hash(uint32_t v);
uint32_t or_bounce_hash(uint32_t seed, uint32_t rid, uint32_t bounce, uint32_t k);
int or_bounce(const float* ray8, float t, const float* tri9, uint32_t seed,
              uint32_t rid, uint32_t bounce, float* out8);

/* Learned-proposal seeds (not in the paper): the frontier of depth D in
   pre-order (slot child/count and box), and the seeded closest-hit
   traversal (see oracle.c). */
int or_bvh_frontier(const OrBvh* b, int D, int32_t* fchild, int32_t* fcount, float* fbox,
                    uint8_t* cls);
int or_trace_seeded(const OrBvh* b, const float* tris, const float* rays, int64_t n,
                    int cull, int skip_bits, int stride, int leaf_min, const int32_t* cls,
                    const int32_t* fchild, const int32_t* fcount, const float* fbox, int nf,
                    float* hit_t, int32_t* hit_id, float* hit_uv, uint32_t* counts);

/* 4-wide view of the binary tree (Sec. 3.2.4 / Fig. 5 use 4-wide nodes):
   a 4-wide node made from binary node n holds, in order, for each child
   slot c of n, the two child slots of c if c is inner, else c itself.
   Returns the number of 4-wide nodes (pre-order, root 0).  Export: per node
   its child count and per child slot (binary parent, child index, 4-wide
   node of an inner child or -1). */
int64_t or_bvh_wide(OrBvh* b);
void or_bvh_wide_export(const OrBvh* b, int32_t* n, int64_t* p, int32_t* c, int64_t* next);
/* Alg. 4 on the 4-wide tree (children ordered by entry distance, ties by
   position); arguments as or_trace_range (builds the 4-wide view). */
int or_trace4_range(OrBvh* b, const float* tris, const float* rays, int64_t r_begin,
                    int64_t r_end, int mode, int cull, int skip_bits, int stride, int leaf_min,
                    float* hit_t, int32_t* hit_id, float* hit_uv, uint32_t* counts,
                    uint32_t* mask_tests);

/* Single ray-triangle test and slab test, exposed for pins. */
int or_ray_tri(const float* ray8, const float* tri9, float tcur, float* t,
               float* u, float* v);
int or_slab(const float* ray8, const float* box6, float tcur, float* tn,
            float* tf);
int or_cell(float p, float lo, float hi, int R);
int or_cell_t(float t, float o, float d, float lo, float hi, int R);
int or_cell_at(float t, float o, float d, float lo, float hi, int R);

#ifdef __cplusplus
}
#endif
#endif
